// Plan serialization: a plan written to bytes and read back (a cache of the
// host analysis), its digest, and the layout fingerprint that refuses
// buffers from builds with another plan layout.
#include <cstdint>
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "slu_internal.hpp"

using namespace slu;

// Plan serialization (caching the host analysis).  A plan is plain host
// arrays and scalars; SLU_PLAN_FIELDS lists every field the factorization
// and the solves read, in one fixed order, and drives the byte format, the
// digest and a layout fingerprint (field names and element sizes), so a
// field added to, removed from or retyped in slu_plan changes the
// fingerprint and old buffers are refused.  analyze_ms and phase_ms (timings)
// travel in the header, outside the digest; the device mirror is never written.

namespace slu {
namespace {

#define SLU_PLAN_FIELDS(X)                                                    \
    X(opts) X(n) X(nnz_a) X(nnz_sym)                                          \
    X(a_colptr) X(a_rowidx) X(a_rowptr) X(a_colidx) X(a_vpos) X(a_ci)         \
    X(f_colptr) X(f_rowidx) X(flops) X(flops_cls)                             \
    X(blockptr) X(ptr) X(p) X(samples) X(maxb) X(regular_block) X(seg)       \
    X(row_seg) X(rowblk)                                                      \
    X(blocks) X(bnnz) X(diagblk) X(lcolptr) X(lrow) X(dpos) X(sched) X(sgrp)  \
    X(lr_ptr) X(lr_pos) X(lr_col) X(ur_ptr) X(ur_pos) X(ur_col)               \
    X(ne_off) X(ne_col) X(storage) X(ndense) X(level) X(nlevels)              \
    X(getrf_off) X(gessm_off) X(tstrf_off) X(tgt_off) X(getrf)                \
    X(gd_off) X(gs_off) X(gd) X(gs) X(dv_off) X(dn_off) X(dv_pos) X(dn_pos)   \
    X(gessm) X(tstrf) X(tgt) X(srcoff) X(src)                                 \
    X(gm_off) X(gm_task) X(gm_src) X(gm_mask) X(gm_moff) X(gg_off) X(gg_tgt) X(gg_srcoff) X(gg_src) \
    X(gm_mid) X(gg_mid) X(ps_off) X(ps_task) X(pv_off) X(pv_task)             \
    X(woff) X(wsize) X(inv_maxb) X(inv_off) X(inv_task) X(pd_off) X(pd_task)  \
    X(pg_off) X(pg_gessm) X(pg_tstrf) X(pg_goff) X(pg_toff)                   \
    X(sp_off) X(sp_pairs) X(sp_poff) X(sd_pair0) X(part_elems)                \
    X(lrow_off) X(urow_off) X(ucol_off) X(lcol_off)                           \
    X(lrow_blk) X(urow_blk) X(ucol_blk) X(lcol_blk) X(a2s) X(f2s)

// Changes whenever the meaning of a field changes without a change of layout.
constexpr uint32_t kPlanFormat = 4;
constexpr char kPlanMagic[8] = {'S', 'L', 'U', 'P', 'L', 'A', 'N', 0};
constexpr uint32_t kEndian = 0x01020304u;

// 64-bit multiply-xor hash over 8-byte words (FNV-1a's offset and prime,
// one multiply per word), with a splitmix64-style finalizer.  A checksum,
// not a cryptographic hash.  Chunking of the input does not matter.
struct Hasher {
    uint64_t h = 0xcbf29ce484222325ull, acc = 0, total = 0;
    int nacc = 0;
    static constexpr uint64_t kPrime = 0x100000001b3ull;
    void raw(const void *p, size_t len) {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        total += len;
        while (len && nacc) {
            acc |= (uint64_t)*b++ << (8 * nacc);
            --len;
            if (++nacc == 8) {
                h = (h ^ acc) * kPrime;
                acc = 0;
                nacc = 0;
            }
        }
        for (; len >= 8; len -= 8, b += 8) {
            uint64_t w;
            std::memcpy(&w, b, 8);
            h = (h ^ w) * kPrime;
        }
        for (; len; --len) acc |= (uint64_t)*b++ << (8 * nacc++);
    }
    uint64_t done() const {
        uint64_t x = h;
        if (nacc) x = (x ^ acc) * kPrime;
        x = (x ^ total) * kPrime;
        x ^= x >> 30;
        x *= 0xbf58476d1ce4e5b9ull;
        x ^= x >> 27;
        x *= 0x94d049bb133111ebull;
        return x ^ (x >> 31);
    }
};

struct Counter {
    int64_t bytes = 0;
    void raw(const void *, size_t len) { bytes += (int64_t)len; }
};

struct Writer {
    unsigned char *at;
    void raw(const void *p, size_t len) {
        if (len) std::memcpy(at, p, len);
        at += len;
    }
};

struct Reader {
    const unsigned char *at, *end;
    bool ok = true;
    size_t left() const { return (size_t)(end - at); }
    void raw(void *p, size_t len) {
        if (!ok || len > left()) {
            ok = false;
            return;
        }
        if (len) std::memcpy(p, at, len);
        at += len;
    }
};

template <class S, class T>
typename std::enable_if<std::is_arithmetic<T>::value>::type put(S &s, const T &x) {
    s.raw(&x, sizeof(T));
}
template <class S>
void put(S &s, const slu_opts &o) {     // member by member: no padding bytes
    put(s, o.blocking); put(s, o.regular_block); put(s, o.sample_points);
    put(s, o.step); put(s, o.max_num); put(s, o.stride); put(s, o.b_min);
    put(s, o.precision); put(s, o.dense_threshold); put(s, o.pivot_perturb);
    put(s, o.pivot_tau_rel); put(s, o.refine_tol); put(s, o.refine_max_iter);
    put(s, o.wait_budget_ms); put(s, o.tc_passes);
}
template <class S, class T, class A>
void put(S &s, const std::vector<T, A> &v) {   // element types have no padding
    const int64_t c = (int64_t)v.size();
    put(s, c);
    s.raw(v.data(), v.size() * sizeof(T));
}
template <class S, class T, size_t N>
void put(S &s, const T (&a)[N]) {
    for (const T &e : a) put(s, e);
}

template <class T>
typename std::enable_if<std::is_arithmetic<T>::value>::type get(Reader &r, T &x) {
    r.raw(&x, sizeof(T));
}
void get(Reader &r, slu_opts &o) {
    get(r, o.blocking); get(r, o.regular_block); get(r, o.sample_points);
    get(r, o.step); get(r, o.max_num); get(r, o.stride); get(r, o.b_min);
    get(r, o.precision); get(r, o.dense_threshold); get(r, o.pivot_perturb);
    get(r, o.pivot_tau_rel); get(r, o.refine_tol); get(r, o.refine_max_iter);
    get(r, o.wait_budget_ms); get(r, o.tc_passes);
}
template <class T, class A>
void get(Reader &r, std::vector<T, A> &v) {
    int64_t c = 0;
    get(r, c);
    if (!r.ok || c < 0 || (uint64_t)c > r.left() / sizeof(T)) {
        r.ok = false;
        return;
    }
    v.resize((size_t)c);
    r.raw(v.data(), (size_t)c * sizeof(T));
}
template <class T, size_t N>
void get(Reader &r, T (&a)[N]) {
    for (T &e : a) get(r, e);
}

template <class T> uint64_t elem_size(const T &) { return sizeof(T); }
template <class T, class A>
uint64_t elem_size(const std::vector<T, A> &) { return 1000 + sizeof(T); }
template <class T, size_t N> uint64_t elem_size(const T (&a)[N]) {
    return N * 1000000 + elem_size(a[0]);
}

template <class S>
void put_fields(S &s, const slu_plan &P) {
#define SLU_PUT(f) put(s, P.f);
    SLU_PLAN_FIELDS(SLU_PUT)
#undef SLU_PUT
}

uint64_t fingerprint() {
    slu_plan P;
    Hasher h;
    uint64_t sz;
#define SLU_FP(f)                 \
    h.raw(#f, sizeof(#f));        \
    sz = elem_size(P.f);          \
    h.raw(&sz, sizeof(sz));
    SLU_PLAN_FIELDS(SLU_FP)
#undef SLU_FP
    return h.done();
}

uint64_t payload_digest(const slu_plan &P) {
    Hasher h;
    put_fields(h, P);
    return h.done();
}

struct Header {
    char magic[8];
    uint32_t format, endian;
    uint64_t fingerprint, digest;
    int64_t payload;
    double analyze_ms;
    double phase_ms[SLU_PHASE_COUNT];
};
static_assert(sizeof(Header) == 48 + 8 * SLU_PHASE_COUNT, "serialized header layout");

}  // namespace
}  // namespace slu

extern "C" slu_status slu_plan_digest(const slu_plan *P, uint64_t *digest) {
    if (!P || !digest) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    *digest = payload_digest(*P);
    return SLU_OK;
}

extern "C" slu_status slu_plan_serialize(const slu_plan *P, void *buf,
                                         int64_t *size) {
    if (!P || !size) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    Counter c;
    put_fields(c, *P);
    const int64_t need = (int64_t)sizeof(Header) + c.bytes;
    if (!buf) {
        *size = need;
        return SLU_OK;
    }
    if (*size < need) {
        const int64_t have = *size;
        *size = need;
        return fail(SLU_ERR_INVALID_ARG, "buffer of " + std::to_string(have) +
                                             " bytes, the plan needs " +
                                             std::to_string(need));
    }
    Header hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kPlanMagic, sizeof(hd.magic));
    hd.format = kPlanFormat;
    hd.endian = kEndian;
    hd.fingerprint = fingerprint();
    hd.digest = payload_digest(*P);
    hd.payload = c.bytes;
    hd.analyze_ms = P->analyze_ms;
    std::memcpy(hd.phase_ms, P->phase_ms, sizeof(hd.phase_ms));
    unsigned char *b = static_cast<unsigned char *>(buf);
    std::memcpy(b, &hd, sizeof(hd));
    Writer w{b + sizeof(hd)};
    put_fields(w, *P);
    *size = need;
    return SLU_OK;
}

extern "C" slu_status slu_plan_deserialize(const void *buf, int64_t size,
                                           slu_plan **out) {
    if (!buf || !out) return fail(SLU_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    Header hd;
    if (size < (int64_t)sizeof(hd))
        return fail(SLU_ERR_INVALID_ARG, "buffer shorter than a plan header");
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kPlanMagic, sizeof(hd.magic)) != 0)
        return fail(SLU_ERR_INVALID_ARG, "not a serialized plan");
    if (hd.endian != kEndian)
        return fail(SLU_ERR_NOT_SUPPORTED, "plan written with another byte order");
    if (hd.format != kPlanFormat || hd.fingerprint != fingerprint())
        return fail(SLU_ERR_NOT_SUPPORTED,
                    "plan written by an incompatible build of the library");
    if (hd.payload != size - (int64_t)sizeof(hd))
        return fail(SLU_ERR_INVALID_ARG, "plan buffer size does not match its header");
    slu_plan *P = new (std::nothrow) slu_plan();
    if (!P) return fail(SLU_ERR_OUT_OF_MEMORY, "plan allocation");
    try {
        const unsigned char *b = static_cast<const unsigned char *>(buf);
        Reader r{b + sizeof(hd), b + size};
#define SLU_GET(f) get(r, P->f);
        SLU_PLAN_FIELDS(SLU_GET)
#undef SLU_GET
        const int64_t n = P->n;
        const bool shape_ok =
            r.ok && r.at == r.end && n >= 0 &&
            (int64_t)P->a_colptr.size() == n + 1 &&
            (int64_t)P->f_colptr.size() == n + 1 &&
            (int64_t)P->blockptr.size() == n + 1 &&
            (int64_t)P->ptr.size() == (int64_t)P->p + 1 &&
            (int64_t)P->diagblk.size() == P->p &&
            (int64_t)P->level.size() == P->p &&
            (int64_t)P->a2s.size() == P->nnz_a &&
            (int64_t)P->f2s.size() == P->f_colptr[n];
        if (!shape_ok) {
            delete P;
            return fail(SLU_ERR_INVALID_ARG, "truncated or inconsistent plan buffer");
        }
        if (payload_digest(*P) != hd.digest) {
            delete P;
            return fail(SLU_ERR_INVALID_ARG, "plan buffer checksum mismatch");
        }
        const slu_status st = slu_plan_check(P);
        if (st != SLU_OK) {
            delete P;
            return st;
        }
    } catch (const std::exception &e) {
        delete P;
        return fail(SLU_ERR_OUT_OF_MEMORY,
                    std::string("host allocation in deserialize: ") + e.what());
    }
    P->analyze_ms = hd.analyze_ms;
    std::memcpy(P->phase_ms, hd.phase_ms, sizeof(hd.phase_ms));
    *out = P;
    return SLU_OK;
}
