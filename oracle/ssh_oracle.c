/*
 * ssh_oracle.c -- plain FP64 CPU oracle for the SSH index and query path
 * (Luo & Shrivastava, arXiv:1610.07328).
 *
 * TEST INFRASTRUCTURE: used only by tests/, the smoke check and the benchmark's
 * CPU-baseline leg. It shares no code with the CUDA library. Each function
 * follows the paper's definition step by step; see ssh_oracle.h for the
 * sections, equations and readings each one follows.
 *
 * Compile with -ffp-contract=off (no fused multiply-add).
 */
#include "ssh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Published constants of Philox4x32 (Salmon et al., SC'11, Sec. 5). */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u
#define PHILOX_WEYL_B 0xBB67AE85u

void ssh_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* the key is bumped between rounds */
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double ssh_oracle_uniform(uint32_t x) {
    double top23 = (double)(x >> 9);
    return (top23 + 0.5) * (1.0 / 8388608.0); /* 2^-23 */
}

/* Domain tags keep the filter draws and the minhash draws on disjoint counters. */
#define TAG_FILTER 0x46494C54u /* "FILT" */
#define TAG_CWS 0x43575331u    /* "CWS1" */
#define TAG_SRP 0x53525031u    /* "SRP1" */

static void seed_key(uint64_t seed, uint32_t key[2]) {
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
}

/* Sec. 4.1, "the entries of r are i.i.d. normal": Box-Muller on two uniforms of
 * the Philox block with counter (p, 0, FILT, 0); entry 2p takes the cosine
 * branch, entry 2p+1 the sine branch. */
void ssh_oracle_filter(uint64_t seed, int W, float* r_out) {
    uint32_t key[2];
    seed_key(seed, key);
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < W; ++j) {
        uint32_t ctr[4] = {(uint32_t)(j / 2), 0u, TAG_FILTER, 0u};
        uint32_t blk[4];
        ssh_oracle_philox4x32_10(ctr, key, blk);
        double u1 = ssh_oracle_uniform(blk[0]);
        double u2 = ssh_oracle_uniform(blk[1]);
        double radius = sqrt(-2.0 * log(u1));
        double angle = two_pi * u2;
        double z = (j % 2 == 0) ? radius * cos(angle) : radius * sin(angle);
        r_out[j] = (float)z;
    }
}

/* The SRP baseline (Sec. 5.2, Table 2): projection j of length m has i.i.d.
 * normal entries, Box-Muller on the Philox block with counter (i/2, j, SRP1, m)
 * (cosine branch for even i, sine for odd i), each rounded once to FP32. */
void ssh_oracle_srp_projection(uint64_t seed, int m, int j, float* r_out) {
    uint32_t key[2];
    seed_key(seed, key);
    const double two_pi = 6.283185307179586476925286766559;
    for (int i = 0; i < m; ++i) {
        uint32_t ctr[4] = {(uint32_t)(i / 2), (uint32_t)j, TAG_SRP, (uint32_t)m};
        uint32_t blk[4];
        ssh_oracle_philox4x32_10(ctr, key, blk);
        double u1 = ssh_oracle_uniform(blk[0]);
        double u2 = ssh_oracle_uniform(blk[1]);
        double radius = sqrt(-2.0 * log(u1));
        double angle = two_pi * u2;
        double z = (i % 2 == 0) ? radius * cos(angle) : radius * sin(angle);
        r_out[i] = (float)z;
    }
}

/* Sign random projections of x over the whole series: bit j = [r_j . x >= 0],
 * the dot product in FP64, summed in index order. */
void ssh_oracle_srp_bits(const float* x, int m, uint64_t seed, int nhash, uint32_t* bits_out) {
    float* r = (float*)malloc(sizeof(float) * (size_t)m);
    for (int j = 0; j < nhash; ++j) {
        ssh_oracle_srp_projection(seed, m, j, r);
        double d = 0.0;
        for (int i = 0; i < m; ++i) d = d + (double)r[i] * (double)x[i];
        bits_out[j] = d >= 0.0 ? 1u : 0u;
    }
    free(r);
}

/* ---------------------------------------------------------------- Sketch */

int ssh_oracle_num_bits(int m, int W, int delta) {
    if (W < 1 || delta < 1 || m < W) return 0;
    return (m - W) / delta + 1;
}

double ssh_oracle_window_dot(const float* x, const float* r, int W, int start) {
    double acc = 0.0;
    for (int j = 0; j < W; ++j) acc = acc + (double)r[j] * (double)x[start + j];
    return acc;
}

void ssh_oracle_sketch(const float* x, int m, const float* r, int W, int delta, uint8_t* bits_out) {
    int nb = ssh_oracle_num_bits(m, W, delta);
    for (int i = 0; i < nb; ++i) {
        double dot = ssh_oracle_window_dot(x, r, W, i * delta);
        bits_out[i] = (dot >= 0.0) ? 1 : 0; /* "+1 : r.X >= 0" */
    }
}

/* --------------------------------------------------------------- Shingle */

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

int ssh_oracle_shingle(const uint8_t* bits, int nb, int n, uint32_t* ids_out, uint32_t* counts_out) {
    if (n < 1 || n > 32 || nb < n) return 0;
    int s = nb - n + 1;
    uint32_t* all = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)s);
    for (int i = 0; i < s; ++i) {
        uint32_t id = 0;
        for (int j = 0; j < n; ++j) id = (id << 1) | (uint32_t)(bits[i + j] & 1u);
        all[i] = id;
    }
    qsort(all, (size_t)s, sizeof(uint32_t), cmp_u32);
    int nnz = 0;
    for (int i = 0; i < s; ++i) {
        if (nnz > 0 && ids_out[nnz - 1] == all[i]) {
            counts_out[nnz - 1] += 1;
        } else {
            ids_out[nnz] = all[i];
            counts_out[nnz] = 1;
            nnz += 1;
        }
    }
    free(all);
    return nnz;
}

/* --------------------------------------------------- Weighted minhash (ICWS) */

/* Natural logarithm of a positive normal double as a fixed sequence of IEEE
 * round-to-nearest operations, so that every machine (and a GPU doing the same
 * operations) gets the same bits: x = 2^e f with f in [sqrt(1/2), sqrt(2))
 * (exact, by the exponent bits), ln f = 2 atanh(s) with s = (f - 1) / (f + 1)
 * and the atanh series s + s^3/3 + ... + s^23/23 (|s| <= 0.1716, so the first
 * omitted term is below 2^-60 of the sum), and ln x = e ln2_hi + (ln f + e ln2_lo)
 * with Cody and Waite's split of ln 2 (the hi part has 11 trailing zero bits,
 * so e ln2_hi is exact). Accurate to a few ulp. Returns NaN outside its domain. */
#define LN2_HI 6.93147180369123816490e-01 /* 0x3FE62E42FEE00000 */
#define LN2_LO 1.90821492927058770002e-10 /* 0x3DEA39EF35793C76 */

double ssh_oracle_ln(double x) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int ex = (int)((bits >> 52) & 0x7FF);
    if (!(x > 0.0) || ex == 0 || ex == 0x7FF) return NAN;
    int e = ex - 1023;
    uint64_t fb = (bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull; /* f in [1, 2) */
    double f;
    memcpy(&f, &fb, sizeof f);
    if (f > 1.41421356237309504880) { /* f / 2, exact */
        fb = (fb & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull;
        memcpy(&f, &fb, sizeof f);
        e += 1;
    }
    double s = (f - 1.0) / (f + 1.0);
    double z = s * s;
    double p = 1.0 / 23.0;
    p = 1.0 / 21.0 + z * p;
    p = 1.0 / 19.0 + z * p;
    p = 1.0 / 17.0 + z * p;
    p = 1.0 / 15.0 + z * p;
    p = 1.0 / 13.0 + z * p;
    p = 1.0 / 11.0 + z * p;
    p = 1.0 / 9.0 + z * p;
    p = 1.0 / 7.0 + z * p;
    p = 1.0 / 5.0 + z * p;
    p = 1.0 / 3.0 + z * p;
    double s2 = s + s;
    double lnf = s2 + s2 * (z * p);
    double de = (double)e;
    return de * LN2_HI + (lnf + de * LN2_LO);
}

void ssh_oracle_cws_draw(uint64_t seed, uint32_t j, uint32_t k, double* r, double* c, double* beta) {
    uint32_t key[2];
    seed_key(seed, key);
    uint32_t ctr0[4] = {k, j, TAG_CWS, 0u};
    uint32_t ctr1[4] = {k, j, TAG_CWS, 1u};
    uint32_t b0[4], b1[4];
    ssh_oracle_philox4x32_10(ctr0, key, b0);
    ssh_oracle_philox4x32_10(ctr1, key, b1);
    double u1 = ssh_oracle_uniform(b0[0]);
    double u2 = ssh_oracle_uniform(b0[1]);
    double u3 = ssh_oracle_uniform(b0[2]);
    double u4 = ssh_oracle_uniform(b0[3]);
    double u5 = ssh_oracle_uniform(b1[0]);
    *r = -ssh_oracle_ln(u1 * u2);    /* Gamma(2,1) as the sum of two Exp(1) */
    *c = -ssh_oracle_ln(u3 * u4);    /* Gamma(2,1) */
    *beta = u5;                      /* U(0,1) */
}

double ssh_oracle_cws_log_a(double r, double c, double beta, uint32_t S, double* t_out) {
    double ln_s = ssh_oracle_ln((double)S);
    double t = floor(ln_s / r + beta);
    double ln_a = ssh_oracle_ln(c) - r * ((t - beta) + 1.0);
    *t_out = t;
    return ln_a;
}

void ssh_oracle_cws(uint64_t seed, int nhash, const uint32_t* ids, const uint32_t* counts, int nnz,
                    uint32_t* kstar, uint32_t* tstar) {
    for (int j = 0; j < nhash; ++j) {
        double best = INFINITY;
        uint32_t best_k = 0, best_t = 0;
        for (int e = 0; e < nnz; ++e) { /* ids ascending: strict < keeps the smaller k on ties */
            double r, c, beta, t;
            ssh_oracle_cws_draw(seed, (uint32_t)j, ids[e], &r, &c, &beta);
            double ln_a = ssh_oracle_cws_log_a(r, c, beta, counts[e], &t);
            if (ln_a < best) {
                best = ln_a;
                best_k = ids[e];
                best_t = (uint32_t)t;
            }
        }
        kstar[j] = best_k;
        tstar[j] = best_t;
    }
}

/* ------------------------------------------------------------ Bucket keys */

/* splitmix64 output finalizer (Steele, Lea & Flood, OOPSLA'14; Stafford's mix13). */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t ssh_oracle_bucket_key(uint64_t seed, int l, int K, const uint32_t* kstar, const uint32_t* tstar) {
    uint64_t h = seed ^ (0x9E3779B97F4A7C15ull * (uint64_t)(l + 1));
    for (int i = 0; i < K; ++i) {
        int j = l * K + i;
        uint64_t v = ((uint64_t)kstar[j] << 32) | (uint64_t)tstar[j];
        h = mix64(h ^ v);
    }
    return h;
}

/* A faster weighted minhash among those the paper cites (Sec. 2.3): densified
 * one-permutation hashing of the copies. The integer weighted set {(k, S_k)} is
 * read as the plain set of copies (k, c), c = 1 .. S_k, whose Jaccard similarity
 * is the weighted Jaccard of the counts. Copy (k, c) has v = mix64(seed ^ D1 ^
 * (k << 32 | c)), goes to bin floor((v >> 32) * nhash / 2^32) and has value
 * low32(mix64(v)); each bin keeps its copy of smallest (value, k, c). An empty
 * bin i takes the bin of the first non-empty j_t = floor((mix64(seed ^ D2 ^
 * (i << 32 | t)) >> 32) * nhash / 2^32), t = 0, 1, ... (optimal densification),
 * or, after 64 nhash attempts, the first non-empty bin after i. Hash i is (k, c)
 * of the copy it ends with; an empty set gives (2^32 - 1, 0) everywhere. */
#define DOPH_BIN 0xD0F1B1A5C0FFEE01ull
#define DOPH_FILL 0xDE45E1F1A11B0B02ull

static uint32_t doph_scale(uint64_t v, int nhash) { return (uint32_t)(((v >> 32) * (uint64_t)nhash) >> 32); }

void ssh_oracle_doph(uint64_t seed, int nhash, const uint32_t* ids, const uint32_t* counts, int nnz,
                     uint32_t* kstar, uint32_t* tstar) {
    uint64_t* bins = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nhash);
    for (int i = 0; i < nhash; ++i) bins[i] = UINT64_MAX;
    for (int e = 0; e < nnz; ++e) {
        for (uint32_t c = 1; c <= counts[e]; ++c) {
            uint64_t pack = ((uint64_t)ids[e] << 32) | (uint64_t)c;
            uint64_t v = mix64(seed ^ DOPH_BIN ^ pack);
            uint32_t b = doph_scale(v, nhash);
            uint64_t key = ((uint64_t)(uint32_t)mix64(v) << 32) | ((uint64_t)ids[e] << 16) | (uint64_t)c;
            if (key < bins[b]) bins[b] = key;
        }
    }
    for (int i = 0; i < nhash; ++i) {
        uint64_t key = bins[i];
        if (key == UINT64_MAX && nnz > 0) {
            long long tries = 64LL * nhash;
            for (long long t = 0; t < tries && key == UINT64_MAX; ++t) {
                uint32_t j = doph_scale(mix64(seed ^ DOPH_FILL ^ (((uint64_t)i << 32) | (uint64_t)t)), nhash);
                key = bins[j];
            }
            for (int d = 1; d < nhash && key == UINT64_MAX; ++d) key = bins[(i + d) % nhash];
        }
        if (key == UINT64_MAX) {
            kstar[i] = 0xFFFFFFFFu;
            tstar[i] = 0u;
        } else {
            kstar[i] = (uint32_t)((key >> 16) & 0xFFFFu);
            tstar[i] = (uint32_t)(key & 0xFFFFu);
        }
    }
    free(bins);
}

int ssh_oracle_hash_series(const float* x, int m, const float* r, int W, int delta, int n,
                           uint64_t seed, int K, int L, uint32_t* kstar, uint32_t* tstar) {
    int nb = ssh_oracle_num_bits(m, W, delta);
    if (nb < n) return -1;
    uint8_t* bits = (uint8_t*)malloc((size_t)nb);
    uint32_t* ids = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nb);
    uint32_t* counts = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)nb);
    ssh_oracle_sketch(x, m, r, W, delta, bits);
    int nnz = ssh_oracle_shingle(bits, nb, n, ids, counts);
    ssh_oracle_cws(seed, K * L, ids, counts, nnz, kstar, tstar);
    free(bits);
    free(ids);
    free(counts);
    return nnz;
}

/* ------------------------------------------------------------------- DTW */

int ssh_oracle_band_radius(float band, int m) {
    if (!(band > 0.0f)) return 0;
    double rb = floor((double)band * (double)m);
    if (rb > (double)(m - 1)) rb = (double)(m - 1);
    return (int)rb;
}

double ssh_oracle_dtw(const float* a, const float* b, int m, int rb) {
    /* Two rows of the m x m table; cells outside the band |i - j| <= rb are +inf. */
    double* prev = (double*)malloc(sizeof(double) * (size_t)m);
    double* cur = (double*)malloc(sizeof(double) * (size_t)m);
    for (int j = 0; j < m; ++j) prev[j] = INFINITY;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) cur[j] = INFINITY;
        int j_lo = i - rb < 0 ? 0 : i - rb;
        int j_hi = i + rb > m - 1 ? m - 1 : i + rb;
        for (int j = j_lo; j <= j_hi; ++j) {
            double diff = (double)a[i] - (double)b[j];
            double cost = diff * diff;
            if (i == 0 && j == 0) {
                cur[j] = cost;
                continue;
            }
            double best = INFINITY;
            if (i > 0 && prev[j] < best) best = prev[j];                 /* D(i-1, j)   */
            if (j > 0 && cur[j - 1] < best) best = cur[j - 1];           /* D(i, j-1)   */
            if (i > 0 && j > 0 && prev[j - 1] < best) best = prev[j - 1]; /* D(i-1, j-1) */
            cur[j] = cost + best;
        }
        double* tmp = prev;
        prev = cur;
        cur = tmp;
    }
    double out = prev[m - 1];
    free(prev);
    free(cur);
    return out;
}

double ssh_oracle_lb_keogh(const float* q, const float* c, int m, int rb) {
    double lb = 0.0;
    for (int i = 0; i < m; ++i) {
        int lo = i - rb < 0 ? 0 : i - rb;
        int hi = i + rb > m - 1 ? m - 1 : i + rb;
        double up = (double)q[lo], low = (double)q[lo];
        for (int t = lo; t <= hi; ++t) {
            if ((double)q[t] > up) up = (double)q[t];
            if ((double)q[t] < low) low = (double)q[t];
        }
        double ci = (double)c[i];
        if (ci > up) {
            double d = ci - up;
            lb = lb + d * d;
        } else if (ci < low) {
            double d = ci - low;
            lb = lb + d * d;
        }
    }
    return lb;
}

double ssh_oracle_lb_kim_fl(const float* q, const float* c, int m) {
    double d0 = (double)q[0] - (double)c[0];
    double lb = d0 * d0;
    if (m > 1) {
        double d1 = (double)q[m - 1] - (double)c[m - 1];
        lb = lb + d1 * d1;
    }
    return lb;
}

double ssh_oracle_lb_keogh_kim(const float* q, const float* c, int m, int rb) {
    double lb = 0.0;
    for (int i = 0; i < m; ++i) {
        double term;
        if (i == 0 || i == m - 1) {
            double d = (double)q[i] - (double)c[i];
            term = d * d;
        } else {
            int lo = i - rb < 0 ? 0 : i - rb;
            int hi = i + rb > m - 1 ? m - 1 : i + rb;
            double up = (double)q[lo], low = (double)q[lo];
            for (int t = lo; t <= hi; ++t) {
                if ((double)q[t] > up) up = (double)q[t];
                if ((double)q[t] < low) low = (double)q[t];
            }
            double ci = (double)c[i];
            term = 0.0;
            if (ci > up) term = (ci - up) * (ci - up);
            else if (ci < low) term = (ci - low) * (ci - low);
        }
        lb = lb + term;
    }
    return lb;
}

/* (d1, id1) < (d2, id2) in lexicographic order; an empty slot (id -1) is last. */
static int pair_less(double d1, int64_t id1, double d2, int64_t id2) {
    if (id2 < 0) return 1;
    if (d1 != d2) return d1 < d2;
    return id1 < id2;
}

void ssh_oracle_topk_dtw(const float* q, const float* rows, const int64_t* ids, int64_t n, int m,
                         int rb, int k, int64_t* out_ids, double* out_d) {
    for (int s = 0; s < k; ++s) {
        out_ids[s] = -1;
        out_d[s] = INFINITY;
    }
    for (int64_t i = 0; i < n; ++i) {
        double d = ssh_oracle_dtw(q, rows + (size_t)i * (size_t)m, m, rb);
        int64_t id = ids[i];
        int pos = k; /* insertion into the sorted list of the k best pairs */
        while (pos > 0 && pair_less(d, id, out_d[pos - 1], out_ids[pos - 1])) pos -= 1;
        if (pos >= k) continue;
        for (int s = k - 1; s > pos; --s) {
            out_d[s] = out_d[s - 1];
            out_ids[s] = out_ids[s - 1];
        }
        out_d[pos] = d;
        out_ids[pos] = id;
    }
}
