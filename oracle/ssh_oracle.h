/*
 * ssh_oracle.h -- plain FP64 CPU oracle for the SSH (Sketch, Shingle & Hash)
 * index and query path of Luo & Shrivastava, "SSH (Sketch, Shingle, & Hash)
 * for Indexing Massive-Scale Time Series" (arXiv:1610.07328).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use this code. It shares nothing with the CUDA library: it
 * has its own header, its own Philox, its own key mixing, and it is compiled on
 * its own. Everything is written for clarity, not speed: sequential loops, FP64
 * arithmetic, no blocking and no reordering.
 *
 * All floating-point code is compiled with -ffp-contract=off so that every
 * multiply and add is rounded on its own (no fused multiply-add), exactly as the
 * expressions are written.
 */
#ifndef SSH_ORACLE_H
#define SSH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 block function (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel
 * random numbers: as easy as 1, 2, 3"): 10 rounds of the 4x32 Philox S-box with
 * the published multipliers and Weyl key increments. */
void ssh_oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Uniform in (0,1) from one 32-bit word: ((x >> 9) + 1/2) * 2^-23. The result is
 * an odd multiple of 2^-24, exactly representable in FP32 and FP64, never 0 or 1. */
double ssh_oracle_uniform(uint32_t x);

/* The random filter r of Sec. 4.1 (entries i.i.d. N(0,1)), drawn from `seed` with
 * Box-Muller on Philox uniforms and rounded once to FP32. */
void ssh_oracle_filter(uint64_t seed, int W, float* r_out);
/* SRP baseline: projection j of length m (FP32 normals), and the nhash sign bits of x. */
void ssh_oracle_srp_projection(uint64_t seed, int m, int j, float* r_out);
void ssh_oracle_srp_bits(const float* x, int m, uint64_t seed, int nhash, uint32_t* bits_out);

/* Number of sketch bits N_B = floor((m - W) / delta) + 1, or 0 when m < W. */
int ssh_oracle_num_bits(int m, int W, int delta);

/* Sec. 4.1: bit i = 1 iff r . x[i*delta .. i*delta + W - 1] >= 0, for i < N_B.
 * The dot product is summed in FP64, j = 0 .. W-1 in order. bits_out[i] is 0 or 1. */
void ssh_oracle_sketch(const float* x, int m, const float* r, int W, int delta, uint8_t* bits_out);

/* The FP64 dot product behind one sketch bit (for tests). */
double ssh_oracle_window_dot(const float* x, const float* r, int W, int start);

/* Sec. 4.2 / Eq. (set): the weighted set of all length-n substrings of the bit
 * string. Shingle id = bits[i..i+n-1] read as an n-bit integer, first bit most
 * significant. Writes the distinct ids in ascending order with their counts and
 * returns how many there are (0 when nb < n). ids_out/counts_out hold nb entries. */
int ssh_oracle_shingle(const uint8_t* bits, int nb, int n, uint32_t* ids_out, uint32_t* counts_out);

/* Natural logarithm used by the weighted-minhash draws: a fixed sequence of IEEE
 * FP64 operations (exponent split, atanh series, Cody-Waite ln 2), so the draws
 * are the same bits on every machine. Positive normal x; NaN otherwise. */
double ssh_oracle_ln(double x);

/* The random draws of one weighted-minhash function j for one shingle id k (Ioffe
 * 2010, "Improved Consistent Sampling"): r ~ Gamma(2,1), c ~ Gamma(2,1),
 * beta ~ U(0,1), all from Philox keyed on (seed) with counter (k, j, tag, block):
 * r = -ln(u1 u2), c = -ln(u3 u4), beta = u5 with ln = ssh_oracle_ln. */
void ssh_oracle_cws_draw(uint64_t seed, uint32_t j, uint32_t k, double* r, double* c, double* beta);

/* ln a for one (j, k, S): t = floor(ln S / r + beta), ln a = ln c - r * ((t - beta) + 1),
 * every logarithm by ssh_oracle_ln.
 * Writes t to *t_out. */
double ssh_oracle_cws_log_a(double r, double c, double beta, uint32_t S, double* t_out);

/* Sec. 4.3: weighted minhash of a weighted set (ids ascending, counts > 0) for the
 * hash functions j = 0 .. nhash-1. (kstar, tstar) = the (k, t_k) of the smallest
 * ln a_k; equal values go to the smaller k. */
void ssh_oracle_cws(uint64_t seed, int nhash, const uint32_t* ids, const uint32_t* counts, int nnz,
                    uint32_t* kstar, uint32_t* tstar);

/* 64-bit bucket key of table l from the K hashes j = l*K .. l*K + K - 1 (a
 * splitmix64-finalizer fold; used only to compare with the library's keys, the
 * oracle's own tables compare the K-tuples themselves). */
uint64_t ssh_oracle_bucket_key(uint64_t seed, int l, int K, const uint32_t* kstar, const uint32_t* tstar);
/* Densified one-permutation weighted minhash of a weighted set (ids < 2^16, counts < 2^16). */
void ssh_oracle_doph(uint64_t seed, int nhash, const uint32_t* ids, const uint32_t* counts, int nnz,
                     uint32_t* kstar, uint32_t* tstar);

/* Sec. 4.1-4.3 for one series: sketch, shingle, weighted minhash. kstar/tstar hold
 * K*L entries. Returns the number of distinct shingles, or -1 if the series is too
 * short to give one shingle. */
int ssh_oracle_hash_series(const float* x, int m, const float* r, int W, int delta, int n,
                           uint64_t seed, int K, int L, uint32_t* kstar, uint32_t* tstar);

/* Sakoe-Chiba radius r_b = floor(band * m), with band taken as the FP32 value given. */
int ssh_oracle_band_radius(float band, int m);

/* Sec. 2.1: DTW by dynamic programming over the m x m grid restricted to |i - j| <= rb,
 * cell cost (a_i - b_j)^2, D(i,j) = cost + min(D(i-1,j), D(i,j-1), D(i-1,j-1)),
 * result D(m-1, m-1) (sum of squared costs along the best path, no square root). */
double ssh_oracle_dtw(const float* a, const float* b, int m, int rb);

/* LB_Keogh of candidate c against the envelope of query q with radius rb:
 * U_i = max q[i-rb .. i+rb], L_i = min q[i-rb .. i+rb] (clipped to the series),
 * LB = sum over i of (c_i - U_i)^2 if c_i > U_i, (c_i - L_i)^2 if c_i < L_i, else 0. */
double ssh_oracle_lb_keogh(const float* q, const float* c, int m, int rb);
/* LB_Kim's endpoint bound: every warping path contains the cells (0, 0) and
 * (m-1, m-1), so DTW >= (q_0 - c_0)^2 + (q_{m-1} - c_{m-1})^2 (one cell if m = 1). */
double ssh_oracle_lb_kim_fl(const float* q, const float* c, int m);
/* LB_Keogh whose terms for candidate samples 0 and m-1 are replaced by those two
 * cell costs (each is at least the envelope term it replaces). */
double ssh_oracle_lb_keogh_kim(const float* q, const float* c, int m, int rb);

/* Exact top-k by DTW over rows[0..n) of a row-major [n, m] array (ids[i] names
 * row i): the k smallest (distance, id) pairs in lexicographic order. Unfilled
 * slots get id -1 and distance +inf. */
void ssh_oracle_topk_dtw(const float* q, const float* rows, const int64_t* ids, int64_t n, int m,
                         int rb, int k, int64_t* out_ids, double* out_d);

#ifdef __cplusplus
}
#endif
#endif
