// dtw_wave.cuh -- the banded DTW wavefront (Sec. 2.1, squared costs, Sakoe-Chiba
// radius rb) on a group of lanes per (query, candidate) pair, as a device
// function shared by the DTW kernel and the persistent batch rerank.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssh_internal.cuh"

namespace ssh {
namespace wave {

constexpr unsigned kFull = 0xFFFFFFFFu;

//
// One (query, candidate) pair is handled by a group of G lanes. The band of a
// row has w = 2 rb + 1 cells; it is padded at the front to G*S cells (offset o'
// = o + PAD, PAD = G*S - w, odd) and lane g owns slots o' in [gS, gS + S).
// Cell (i, o) with j = i - rb + o is updated at wave tau = 2 i + o, so one wave
// is one anti-diagonal of the grid (tau = i + j + rb) and holds S/2 independent
// cells per lane: the slots of one parity. Its inputs (i-1, j), (i, j-1),
// (i-1, j-1) are the slots o+1, o-1 (previous wave) and o (two waves ago); the
// slots just outside a lane come from the neighbour lanes by warp shuffle.
// Only the slot right before the first real cell must stay +inf (it is the
// left neighbour of the band's first diagonal); it is forced there once per
// two waves. The band's last diagonal reads +inf from past the last lane.
//
// Samples outside [0, m) read as kPad: a cell with exactly one coordinate
// outside costs ~kPad^2 and never wins, and cells with both coordinates < 0
// cost 0 and start from D = 0, which supplies D(-1,-1) = 0 to cell (0, 0).
//
// The c (candidate) and q (query) windows slide by one sample every two waves;
// the loop is unrolled by the window period U = S/2 + 1 so the slide is a
// renaming of registers, not moves.

// (r0, r1) = (d0 * d0 + c0, d1 * d1 + c1) with one paired FP32 FMA (sm_100+),
// each half rounded once exactly as fmaf: two DTW cells in one issue slot.
__device__ __forceinline__ void sq_add2(float& r0, float& r1, float d0, float d1, float c0, float c1) {
    unsigned long long dd, cc, rr;
    asm("mov.b64 %0, {%1, %2};" : "=l"(dd) : "f"(d0), "f"(d1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c0), "f"(c1));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(rr) : "l"(dd), "l"(cc));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r0), "=f"(r1) : "l"(rr));
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// The pairs [*s_next, b1) of one segment (query qg, staged in q_s by the caller)
// against the band of radius rb, the block's lane groups claiming pairs through
// *s_next; out[slot] = the pair's DTW, or +inf once all its band cells exceed
// bound / shrink (early abandoning). blocks_done (optional) adds the blocks of U
// steps each pair ran.
template <int S, int PMASK>
__device__ __forceinline__ void dtw_wave_pairs(const float* q_s, const float* qg, int m, int rb, int G,
                                               const float* const* pair_b, const int64_t* pair_slot, int64_t b1,
                                               unsigned long long* s_next, float bound, float shrink, float* out,
                                               unsigned long long* blocks_done) {
    constexpr int H = S / 2;
    constexpr int U = H + 1;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 / G;
    const int grp = lane / G, g = lane - grp * G;
    const bool lane_in_group = grp < gpw;
    const unsigned gbits = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (grp * G));
    const int PAD = G * S - (2 * rb + 1);
    const int gmask = (PAD - 1) / S;
    const float mflag = (g == gmask) ? __int_as_float(0x7F800000) : __int_as_float(0xFF800000);
    const float INF = __int_as_float(0x7F800000);
    const int tau_f = 2 * (m - 1) + rb;
    const int s_end = tau_f >> 1;
    const int nblk = (s_end + U) / U;  // ceil((s_end + 1) / U)
    const int s0 = s_end + 1 - nblk * U;
    const int of = rb + PAD;           // slot of the final cell (m-1, m-1)
    const int g_f = of / S, p_f = of - g_f * S;
    // per-lane offsets of the sliding windows: A(s) = s + a_off, B(s) = s + b_off
    const int a_off = -g * H + (PAD - 1) / 2;
    const int b_off = g * H - rb + (1 - PAD) / 2;
    int64_t p = -1;  // the group's pair, -1: none
    int lblk = 0;    // blocks of U steps the group has done on it
    const float* c = qg;
    float D[S], creg[U], qreg[U];
    bool need = lane_in_group;
    while (true) {
        // groups without a pair claim the next one (leader's atomic, shuffled to the group)
        unsigned long long v = ~0ull;
        if (need && g == 0) {
            v = atomicAdd(s_next, 1ull);
            // pairs a reversed LB_Keogh pass cleared are skipped (their distance stays +inf)
            while (v < (unsigned long long)b1 && pair_b[v] == nullptr) v = atomicAdd(s_next, 1ull);
        }
        v = __shfl_sync(kFull, v, lane_in_group ? grp * G : lane);
        if (need) {
            p = (v < (unsigned long long)b1) ? (int64_t)v : -1;
            if (p >= 0) {
                c = pair_b[p];
                lblk = 0;
#pragma unroll
                for (int t = 0; t < S; ++t) D[t] = 0.f;
                if (g == gmask) D[PMASK] = INF;
                // prefill logical cw[t] = c[A(s0) + 1 - t] (t >= 1) and qw[a] = q[B(s0) + a]
                // (a <= H - 2) with the register map of unrolled step u = 0:
                // cw[t] -> creg[t % U], qw[a] -> qreg[a % U]
#pragma unroll
                for (int t = 1; t < U; ++t) {
                    const int ci = s0 + a_off + 1 - t;
                    creg[t] = (ci >= 0 && ci < m) ? __ldg(c + ci) : kPad;
                }
#pragma unroll
                for (int t = 0; t < U; ++t) {
                    const int qi = s0 + b_off + t;
                    qreg[t] = (t < H - 1 && qi >= 0 && qi < m) ? q_s[qi] : kPad;
                }
                creg[0] = 0.f;
            } else {
                c = qg;  // idle: the steps below run on the query itself and are discarded
            }
        }
        if (!__any_sync(kFull, p >= 0)) break;
        const int sbase = s0 + lblk * U;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = sbase + u;
            {   // slide the windows: new cw[0] = c[A(s) + 1], new qw[H-1] = q[B(s) + H - 1]
                const int ci = s + a_off + 1;
                creg[(U - u) % U] = (ci >= 0 && ci < m) ? __ldg(c + ci) : kPad;
                const int qi = s + b_off + H - 1;
                qreg[(H - 1 + u) % U] = (qi >= 0 && qi < m) ? q_s[qi] : kPad;
            }
            // wave tau = 2s: odd slots 2a+1, cell (A - a, B + a), c = cw[a+1], q = qw[a]
            float right = __shfl_down_sync(kFull, D[0], 1);
            if (g == G - 1) right = INF;
            // the cells of a wave are independent: slots 2a+1 and 2a+3 share one paired FMA
#pragma unroll
            for (int a = 0; a < H; a += 2) {
                const int pp = 2 * a + 1;
                const float ur = (pp + 1 < S) ? D[pp + 1] : right;
                const float d = creg[(a + 1 + U - u) % U] - qreg[(a + u) % U];
                const float mn = min3f(ur, D[pp - 1], D[pp]);
                if (a + 1 < H) {
                    const int p1 = pp + 2;
                    const float ur1 = (p1 + 1 < S) ? D[p1 + 1] : right;
                    const float d1 = creg[(a + 2 + U - u) % U] - qreg[(a + 1 + u) % U];
                    const float mn1 = min3f(ur1, D[p1 - 1], D[p1]);
                    sq_add2(D[pp], D[p1], d, d1, mn, mn1);
                } else {
                    D[pp] = fmaf(d, d, mn);
                }
            }
            // wave tau = 2s + 1: even slots 2a, cell (A + 1 - a, B + a), c = cw[a], q = qw[a]
            float left = __shfl_up_sync(kFull, D[S - 1], 1);
            if (g == 0) left = INF;
#pragma unroll
            for (int a = 0; a < H; a += 2) {
                const int pp = 2 * a;
                const float lf = (pp > 0) ? D[pp - 1] : left;
                const float d = creg[(a + U - u) % U] - qreg[(a + u) % U];
                const float mn = min3f(D[pp + 1], lf, D[pp]);
                if (a + 1 < H) {
                    const int p1 = pp + 2;
                    const float d1 = creg[(a + 1 + U - u) % U] - qreg[(a + 1 + u) % U];
                    const float mn1 = min3f(D[p1 + 1], D[p1 - 1], D[p1]);
                    sq_add2(D[pp], D[p1], d, d1, mn, mn1);
                } else {
                    D[pp] = fmaf(d, d, mn);
                }
            }
            D[PMASK] = fmaxf(D[PMASK], mflag);
        }
        ++lblk;
        bool over = false;
        if (bound < INF) {  // uniform over the block
            float lm = INF;
#pragma unroll
            for (int t = 0; t < S; ++t)
                if (g * S + t >= PAD) lm = fminf(lm, D[t]);  // front padding slots are not band cells
            const unsigned bal = __ballot_sync(kFull, lm * shrink > bound);
            over = (bal & gbits) == gbits;
        }
        const bool fin = p >= 0 && lblk == nblk;
        const bool ab = p >= 0 && !fin && over;
        if (fin || ab) {
            float res = INF;
            if (fin) {
#pragma unroll
                for (int t = 0; t < S; ++t)
                    if (t == p_f) res = D[t];
            }
            if (g == g_f) out[pair_slot ? pair_slot[p] : p] = res;
            if (blocks_done && g == 0) atomicAdd(blocks_done, (unsigned long long)lblk);
        }
        need = lane_in_group && (fin || ab);
    }
}

}  // namespace wave
}  // namespace ssh
