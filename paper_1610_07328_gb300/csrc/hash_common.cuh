// hash_common.cuh -- device pieces shared by the two hash kernels: the bucket
// key mix, the certified FP32 evaluation of consistent weighted sampling
// (Sec. 4.3, Ioffe's ICWS) and its exact FP64 recomputation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssh_internal.cuh"

namespace ssh {

// splitmix64 output finalizer (Steele, Lea & Flood, OOPSLA'14).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Algorithm 1 bucket key of table l from its K (k*, t*) pairs.
__device__ __forceinline__ uint64_t bucket_key(uint64_t seed, int l, int K, const uint32_t* kst,
                                               const uint32_t* tst) {
    uint64_t h = seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(l + 1));
    for (int i = 0; i < K; ++i) {
        const int j = l * K + i;
        h = mix64(h ^ (((uint64_t)kst[j] << 32) | (uint64_t)tst[j]));
    }
    return h;
}

// ---------------------------------------------- Sec. 4.3 draws on the device

// Philox4x32-10 (Salmon et al., SC'11): the counter-based generator of every draw.
__host__ __device__ __forceinline__ void philox4x32_10(const uint32_t in[4], uint32_t k0, uint32_t k1,
                                                       uint32_t out[4]) {
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// ((x >> 9) + 1/2) 2^-23: exact in FP32 and FP64, never 0 or 1.
__device__ __forceinline__ double unit23(uint32_t x) {
    return __dmul_rn(__dadd_rn((double)(x >> 9), 0.5), 1.0 / 8388608.0);
}

// Natural logarithm of a positive normal double as one fixed sequence of IEEE
// round-to-nearest operations (so every machine computes the same bits): the
// exponent split x = 2^e f, f in [sqrt(1/2), sqrt(2)); ln f = 2 atanh(s),
// s = (f - 1) / (f + 1), by the series s + s^3/3 + ... + s^23/23 in Horner form;
// ln x = e ln2_hi + (ln f + e ln2_lo) with Cody and Waite's two-part ln 2.
// NaN for zero, negative, subnormal, infinite or NaN x.
__device__ __forceinline__ double ln_fixed(double x) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (!(x > 0.0) || ex == 0 || ex == 0x7FF) return __longlong_as_double(0x7FF8000000000000ll);
    int e = ex - 1023;
    unsigned long long fb = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
    double f = __longlong_as_double((long long)fb);
    if (f > 1.41421356237309504880) {
        fb = (fb & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull;
        f = __longlong_as_double((long long)fb);
        e += 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double z = __dmul_rn(s, s);
    double p = 1.0 / 23.0;
    p = __dadd_rn(1.0 / 21.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 19.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 17.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 15.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 13.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 11.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 9.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 7.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 5.0, __dmul_rn(z, p));
    p = __dadd_rn(1.0 / 3.0, __dmul_rn(z, p));
    const double s2 = __dadd_rn(s, s);
    const double lnf = __dadd_rn(s2, __dmul_rn(s2, __dmul_rn(z, p)));
    const double de = (double)e;
    constexpr double kLn2Hi = 6.93147180369123816490e-01;  // 0x3FE62E42FEE00000
    constexpr double kLn2Lo = 1.90821492927058770002e-10;  // 0x3DEA39EF35793C76
    return __dadd_rn(__dmul_rn(de, kLn2Hi), __dadd_rn(lnf, __dmul_rn(de, kLn2Lo)));
}

constexpr uint32_t kTagCwsDraw = 0x43575331u;  // "CWS1"

// Ioffe's ICWS draws of hash j for shingle k: r = -ln(u1 u2), c = -ln(u3 u4)
// (Gamma(2,1) each), beta = u5 (U(0,1)), from the Philox blocks with counters
// (k, j, CWS1, 0) and (k, j, CWS1, 1) under the key (seed low, seed high).
__device__ __forceinline__ void cws_draw_dev(uint64_t seed, uint32_t j, uint32_t k, double* r, double* beta,
                                             double* lnc) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t c0[4] = {k, j, kTagCwsDraw, 0u};
    const uint32_t c1[4] = {k, j, kTagCwsDraw, 1u};
    uint32_t x[4], y[4];
    philox4x32_10(c0, k0, k1, x);
    philox4x32_10(c1, k0, k1, y);
    *r = -ln_fixed(__dmul_rn(unit23(x[0]), unit23(x[1])));
    const double c = -ln_fixed(__dmul_rn(unit23(x[2]), unit23(x[3])));
    *beta = unit23(y[0]);
    *lnc = ln_fixed(c);
}

// FP64 minhash of hash j with the draws computed here (no tables; any n <= 32):
// t = floor(ln S / r + beta), ln a = ln c - r ((t - beta) + 1), the smallest ln a
// wins, equal values go to the smaller id (ids ascending).
__device__ inline void cws_fp64_otf(const HashArgs& a, int j, const uint32_t* cid, const uint32_t* ccnt, int nnz,
                                    uint32_t* kout, uint32_t* tout) {
    double best = __longlong_as_double(0x7FF0000000000000ll);
    uint32_t bk = 0, bt = 0;
#pragma unroll 1
    for (int e = 0; e < nnz; ++e) {
        const uint32_t k = cid[e];
        double r, beta, lnc;
        cws_draw_dev(a.seed, (uint32_t)j, k, &r, &beta, &lnc);
        const double lns = a.lns64[ccnt[e]];
        const double t = floor(__dadd_rn(__ddiv_rn(lns, r), beta));
        const double la = __dsub_rn(lnc, __dmul_rn(r, __dadd_rn(__dsub_rn(t, beta), 1.0)));
        if (la < best) {
            best = la;
            bk = k;
            bt = (uint32_t)t;
        }
    }
    *kout = bk;
    *tout = bt;
}

// FP64 recomputation of one hash j over the whole weighted set (ids ascending),
// in the order of the definition: t = floor(ln S / r + beta),
// ln a = ln c - r ((t - beta) + 1); the smallest ln a wins, ties to the smaller id.
__device__ inline void cws_fp64(const HashArgs& a, int j, const uint32_t* cid, const uint32_t* ccnt, int nnz,
                                uint32_t* kout, uint32_t* tout) {
    const size_t nk = (size_t)1 << a.n;
    double best = __longlong_as_double(0x7FF0000000000000ll);  // +inf
    uint32_t bk = 0, bt = 0;
#pragma unroll 1
    for (int e = 0; e < nnz; ++e) {
        const uint32_t k = cid[e];
        const double* p = a.p64 + ((size_t)j * nk + k) * 3;
        const double r = p[0], beta = p[1], lnc = p[2];
        const double lns = a.lns64[ccnt[e]];
        const double t = floor(__dadd_rn(__ddiv_rn(lns, r), beta));
        const double la = __dsub_rn(lnc, __dmul_rn(r, __dadd_rn(__dsub_rn(t, beta), 1.0)));
        if (la < best) {
            best = la;
            bk = k;
            bt = (uint32_t)t;
        }
    }
    *kout = bk;
    *tout = bt;
}

constexpr float kTwoPowMinus21 = 4.76837158203125e-07f;  // 8 units in the last place of FP32
constexpr float kRelWidth = 1.0e-6f;                      // >= 8 ulp: also the 1e-6 relative-gap rule

// FP32 evaluation of one repeated shingle (count s >= 2) for one hash, with an
// interval that contains the FP64 value of the definition, tracked as a running
// certified argmin. The interval's half width is 1e-6 * (|ln c| + r (t + 1 - beta)),
// at least 8 ulp of every operand, so it covers the rounding of ln c, r, 1/r,
// ln s and of the three FP32 operations against the exact value.
struct CwsTrack {
    float la, hi, lo1, lo2;
    uint32_t k, t, klo1;
    bool unsure;

    __device__ __forceinline__ void init() {
        la = __int_as_float(0x7F800000);
        hi = 0.f;
        lo1 = la;
        lo2 = la;
        k = 0xFFFFFFFFu;
        t = 0;
        klo1 = 0xFFFFFFFFu;
        unsure = false;
    }

    // p = (r, 1/r, beta, ln c); ls = ln s in FP32; ids arrive in any order
    __device__ __forceinline__ void add(const float4 p, float ls, uint32_t id) {
        const float P = __fmul_ru(ls, p.y);
        const float x = fmaf(ls, p.y, p.z);
        const float ex = __fmul_ru(__fadd_ru(P, 1.0f), kTwoPowMinus21);
        const float f1 = floorf(__fsub_rd(x, ex));
        const float f2 = floorf(__fadd_ru(x, ex));
        unsure |= !(P < 1048576.0f) || (f1 != f2);
        const float v = (f1 + 1.0f) - p.z;
        const float l = fmaf(-p.x, v, p.w);
        const float er = __fmul_ru(__fadd_ru(fabsf(p.w), __fmul_ru(p.x, v)), kRelWidth);
        const float lo = __fsub_rd(l, er), h = __fadd_ru(l, er);
        if (l < la || (l == la && id < k)) {
            la = l;
            hi = h;
            k = id;
            t = (uint32_t)f1;
        }
        if (lo < lo1) {
            lo2 = lo1;
            lo1 = lo;
            klo1 = id;
        } else if (lo < lo2) {
            lo2 = lo;
        }
    }
};

// Combine the exact count-1 winner (by rank; kA = its id, pA its draws) with the
// repeated-shingle track. Returns false when the FP32 decision is not certain.
__device__ __forceinline__ bool cws_decide(bool hasA, uint32_t kA, float4 pA, const CwsTrack& b, uint32_t* ks,
                                           uint32_t* ts) {
    const bool hasB = b.k != 0xFFFFFFFFu;
    if (!hasB) {
        *ks = kA;
        *ts = 0;
        return hasA;
    }
    const float minLoOther = (b.klo1 != b.k) ? b.lo1 : b.lo2;
    if (!hasA) {
        *ks = b.k;
        *ts = b.t;
        return !b.unsure && b.hi < minLoOther;
    }
    const float v = 1.0f - pA.z;  // exact: beta is an odd multiple of 2^-24 in (0,1)
    const float aLa = fmaf(-pA.x, v, pA.w);
    const float er = __fmul_ru(__fadd_ru(fabsf(pA.w), __fmul_ru(pA.x, v)), kRelWidth);
    const float aLo = __fsub_rd(aLa, er), aHi = __fadd_ru(aLa, er);
    const bool winA = (aLa < b.la) || (aLa == b.la && kA < b.k);
    if (winA) {
        *ks = kA;
        *ts = 0;
        return !b.unsure && aHi < b.lo1;
    }
    *ks = b.k;
    *ts = b.t;
    return !b.unsure && b.hi < aLo && b.hi < minLoOther;
}

// Candidates whose FP32 value is the FP64 ln a of the definition rounded once
// (tabulated at index creation): rounding is monotone, so a strictly smaller
// FP32 value means a strictly smaller FP64 value, and only equal FP32 values
// leave the order open (tie).
struct ExactMin {
    float v;
    uint32_t k, t;
    bool tie;
    __device__ __forceinline__ void init() {
        v = __int_as_float(0x7F800000);
        k = 0xFFFFFFFFu;
        t = 0;
        tie = false;
    }
    __device__ __forceinline__ void add(float val, uint32_t id, uint32_t tt) {
        if (val < v) {
            v = val;
            k = id;
            t = tt;
            tie = false;
        } else if (val == v) {
            tie = true;
        }
    }
};

// Winner among the exact group E and the interval-tracked group C (counts above
// the tabulated ones). Returns false when the FP32 decision is not certain
// (then the hash is recomputed in FP64). t = 255 marks a t that was not tabulated.
__device__ __forceinline__ bool exact_decide(const ExactMin& E, const CwsTrack& C, uint32_t* ks, uint32_t* ts) {
    const bool hasE = E.k != 0xFFFFFFFFu, hasC = C.k != 0xFFFFFFFFu;
    if (!hasC) {
        *ks = E.k;
        *ts = E.t;
        return hasE && !E.tie && E.t != 255u;
    }
    const float minLoOtherC = (C.klo1 != C.k) ? C.lo1 : C.lo2;
    if (!hasE) {
        *ks = C.k;
        *ts = C.t;
        return !C.unsure && C.hi < minLoOtherC;
    }
    // E's FP64 value lies within half an ulp of E.v: bracket it by the neighbouring floats
    const float eLo = nextafterf(E.v, __int_as_float(0xFF800000)), eHi = nextafterf(E.v, __int_as_float(0x7F800000));
    if (E.v < C.la || (E.v == C.la && E.k < C.k)) {
        *ks = E.k;
        *ts = E.t;
        return !E.tie && E.t != 255u && !C.unsure && eHi < C.lo1;
    }
    *ks = C.k;
    *ts = C.t;
    return !C.unsure && C.hi < eLo && C.hi < minLoOtherC;
}

}  // namespace ssh
