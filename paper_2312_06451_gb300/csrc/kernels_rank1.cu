// The Grover mixer as a rank-one update, on a state vector over any feasible
// set (all 2^n states, the Hamming-weight-k ones, or whatever set the cost
// vector enumerates).
//
// Sec. 2.4 takes the Grover mixer H_G = |u><u|, u the uniform superposition
// over the feasible set, so e^{-i b H_G} = I + (e^{-i b} - 1)|u><u| changes a
// state only along u (u_x = N^{-1/2}, N the set's size):
//     psi' = phi + d 1,   d = (e^{-i b} - 1) (sum_x phi_x) / N.
// A round is therefore one streaming pass and one scalar: the pass applies the
// previous round's pending d, this round's phase e^{-i g C} and sums the
// result; a one-block kernel turns the sum into the next d.  The vector kept
// in memory is phi_r = e^{-i g_r C} psi_{r-1} (with d_r beside it), which is
// also what the adjoint sweep needs of round r.
//
// Adjoint (Sec. 2.3), with lambda_{p-1} = (C - <C>) psi_{p-1}:
//     beta_r partial:  2 Im[ conj(sum lambda_r) (sum psi_r) ] / N
//     mu_r          =  lambda_r + (e^{+i b_r} - 1) (sum lambda_r / N) 1
//     gamma_r partial: 2 sum_x (C_x - <C>) Im(conj(mu_r,x) phi_r,x)
//     lambda_{r-1}  =  mu_r e^{+i g_r C}
// again one pass and one scalar per round.  Without checkpoints the same pass
// also recovers phi_{r-1} = e^{+i g_r C} phi_r - d_{r-1} in place.
//
// Sums: float32 over a thread's 8 amplitudes of a tile, float64 across the
// tiles a block visits and across the block, then over the blocks in a fixed
// order, so results are bitwise reproducible run to run.
#include "common.cuh"

#include <algorithm>

namespace qg {
namespace {

constexpr int kR1Threads = 256;
constexpr int kR1Pairs = 4;  // float4 (two amplitudes) loads per thread per tile
constexpr int kR1Tile = kR1Threads * kR1Pairs * 2;
constexpr int kR1BlocksPerSM = 8;
constexpr float kTwoPiF = 6.2831853071795864769f;

__device__ __forceinline__ float2 r1_cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 r1_cmul_conj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// e^{-i g C} for a float32 cost: the turn count (g_hi + g_lo) C formed as a
// float pair (exact head product), its integer part removed exactly, the
// remaining fraction of a turn to the hardware sine/cosine.
__device__ __forceinline__ float2 r1_phase_f32(float C, float ghi, float glo) {
    const float th = ghi * C;
    const float te = fmaf(ghi, C, -th);
    const float tl = fmaf(glo, C, te);
    const float f = (th - rintf(th)) + tl;
    float s, c;
    __sincosf(kTwoPiF * f, &s, &c);
    return make_float2(c, -s);
}

// Descriptor (unit) containing global tile t; tb has nd + 1 entries.
__device__ __forceinline__ int r1_find(const uint32_t *__restrict__ tb, int nd, uint32_t t) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block sum of three float64 values, in a fixed order; the result is valid in
// thread 0.  Every thread of the block must call it.
__device__ __forceinline__ void r1_block_sum3(double (&v)[3], double (&red)[3][kR1Threads / 32]) {
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();  // red is free (an earlier sum has been read)
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 3; q++) red[q][w] = v[q];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 3; q++) {
            double s = 0.0;
            for (int i = 0; i < kR1Threads / 32; i++) s += red[q][i];
            v[q] = s;
        }
}

// Cost values of the pair (x, x + 1); `two` false: only x is in range.
template <int COST>
__device__ __forceinline__ void r1_cost_pair(const void *cost, int64_t x, bool two, float &c0, float &c1, int &i0,
                                             int &i1) {
    if constexpr (COST == 0) {
        const float *cf = static_cast<const float *>(cost);
        if (two) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(cf + x));
            c0 = v.x;
            c1 = v.y;
        } else {
            c0 = __ldg(cf + x);
            c1 = 0.f;
        }
        i0 = i1 = 0;
    } else {
        const unsigned char *cb = static_cast<const unsigned char *>(cost);
        if (two) {
            const uchar2 v = __ldg(reinterpret_cast<const uchar2 *>(cb + x));
            i0 = v.x;
            i1 = v.y;
        } else {
            i0 = __ldg(cb + x);
            i1 = 0;
        }
        c0 = (float)i0;
        c1 = (float)i1;
    }
}

template <int COST>
__device__ __forceinline__ float2 r1_phase(const float2 *stab, float C, int ci, const RoundCoef &cf) {
    if constexpr (COST == 1) return stab[ci];
    else return r1_phase_f32(C, cf.g_hi, cf.g_lo);
}

__device__ __forceinline__ float4 r1_ld2(const float2 *p) { return __ldcs(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void r1_st2(float2 *p, float2 a, float2 b) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a.x, a.y, b.x, b.y));
}
// Amplitude pair at even x (x + 1 < N), or the single amplitude x.
__device__ __forceinline__ float4 r1_load_pair(const float2 *p, int64_t x, bool two) {
    if (two) return r1_ld2(p + x);
    const float2 a = p[x];
    return make_float4(a.x, a.y, 0.f, 0.f);
}

// One streaming pass over every tile of every unit of the launch (grid-stride
// over tiles, so block b sees tiles b, b + G, ... and each unit's tiles as one
// run).  Modes, for round r:
//   R1_FWD : phi_r = (phi_{r-1} + d_{r-1}) e^{-i g_r C} (r = 0: the initial
//            state); sums (Re, Im) of phi_r
//   R1_LAST: psi = phi_{p-1} + d_{p-1}; sums C |psi|^2, Re and Im of C psi
//   R1_BWD : lambda_r (stored, or (C - c0) psi_{p-1} for r = p - 1), mu,
//            the gamma_r sum; for r > 0 lambda_{r-1} stored and summed, and
//            without checkpoints phi_{r-1} recovered in place
// Each block writes one (sum, sum, sum) slot per unit it visited: slot
// (b - tile_begin[unit]) mod G.
template <int MODE, int COST>
__global__ void __launch_bounds__(kR1Threads, MODE == R1_BWD ? 3 : 4) r1_pass_kernel(const R1Desc *__restrict__ descs,
                                                             const uint32_t *__restrict__ tb, int nd,
                                                             uint32_t total, int round) {
    __shared__ double red[3][kR1Threads / 32];
    __shared__ float2 stab[COST == 1 ? kPhaseTable : 1];
    const uint32_t G = gridDim.x;
    uint32_t t = blockIdx.x;
    while (t < total) {
        const int di = r1_find(tb, nd, t);
        const R1Desc D = descs[di];
        const uint32_t t_end = tb[di + 1];
        if constexpr (COST == 1)
            if (MODE != R1_LAST) {
                __syncthreads();  // the previous unit's table is no longer read
                for (int i = threadIdx.x; i < kPhaseTable; i += kR1Threads)
                    stab[i] = D.table[round * kPhaseTable + i];
                __syncthreads();
            }
        const int64_t N = D.dim;
        const int64_t ld = D.ld;
        const int p = D.p;
        const RoundCoef cf = D.coef[round];
        const double *sc = D.scal;
        double acc[3] = {0.0, 0.0, 0.0};
        const uint32_t slot = (blockIdx.x + G - tb[di] % G) % G;
        for (; t < t_end; t += G) {
            const int64_t xt = (int64_t)(t - tb[di]) * kR1Tile;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            float4 v[kR1Pairs];
            float c[kR1Pairs][2];
            int ci[kR1Pairs][2];
            if constexpr (MODE == R1_FWD) {
                const bool gen = round == 0 && !D.init;
                const float2 *in = round == 0 ? D.init : D.phi + (D.ckpt ? (int64_t)(round - 1) * ld : 0);
                float2 *out = D.phi + (D.ckpt ? (int64_t)round * ld : 0);
                const float2 dp = round == 0 ? make_float2(0.f, 0.f)
                                             : make_float2((float)sc[4 * (round - 1)], (float)sc[4 * (round - 1) + 1]);
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    const bool two = x + 1 < N;
                    v[j] = make_float4(D.amp0, 0.f, D.amp0, 0.f);
                    c[j][0] = c[j][1] = 0.f;
                    ci[j][0] = ci[j][1] = 0;
                    if (x < N) {
                        if (!gen) v[j] = r1_load_pair(in, x, two);
                        r1_cost_pair<COST>(D.cost, x, two, c[j][0], c[j][1], ci[j][0], ci[j][1]);
                    }
                }
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    if (x >= N) continue;
                    float2 a = make_float2(v[j].x + dp.x, v[j].y + dp.y);
                    a = r1_cmul(a, r1_phase<COST>(stab, c[j][0], ci[j][0], cf));
                    s0 += a.x;
                    s1 += a.y;
                    if (x + 1 < N) {
                        float2 b = make_float2(v[j].z + dp.x, v[j].w + dp.y);
                        b = r1_cmul(b, r1_phase<COST>(stab, c[j][1], ci[j][1], cf));
                        s0 += b.x;
                        s1 += b.y;
                        r1_st2(out + x, a, b);
                    } else {
                        out[x] = a;
                    }
                }
            } else if constexpr (MODE == R1_LAST) {
                const float2 *in = D.phi + (D.ckpt ? (int64_t)(p - 1) * ld : 0);
                const float2 dl = make_float2((float)sc[4 * (p - 1)], (float)sc[4 * (p - 1) + 1]);
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    const bool two = x + 1 < N;
                    v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    c[j][0] = c[j][1] = 0.f;
                    if (x < N) {
                        v[j] = r1_load_pair(in, x, two);
                        r1_cost_pair<COST>(D.cost, x, two, c[j][0], c[j][1], ci[j][0], ci[j][1]);
                    }
                }
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    if (x >= N) continue;
                    float re = v[j].x + dl.x, im = v[j].y + dl.y;
                    float C = c[j][0];
                    s0 = fmaf(C, fmaf(re, re, im * im), s0);
                    s1 = fmaf(C, re, s1);
                    s2 = fmaf(C, im, s2);
                    if (x + 1 < N) {
                        re = v[j].z + dl.x;
                        im = v[j].w + dl.y;
                        C = c[j][1];
                        s0 = fmaf(C, fmaf(re, re, im * im), s0);
                        s1 = fmaf(C, re, s1);
                        s2 = fmaf(C, im, s2);
                    }
                }
            } else {  // R1_BWD
                const bool first = round == p - 1;
                float2 *phi = D.phi + (D.ckpt ? (int64_t)round * ld : 0);
                const float c0 = (float)sc[4 * p];
                const float2 m = make_float2((float)sc[4 * p + 1], (float)sc[4 * p + 2]);
                const float2 dl = make_float2((float)sc[4 * round], (float)sc[4 * round + 1]);
                const float2 dq = round > 0 ? make_float2((float)sc[4 * (round - 1)], (float)sc[4 * (round - 1) + 1])
                                            : make_float2(0.f, 0.f);
                float4 l[kR1Pairs];
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    const bool two = x + 1 < N;
                    v[j] = l[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    c[j][0] = c[j][1] = 0.f;
                    ci[j][0] = ci[j][1] = 0;
                    if (x < N) {
                        v[j] = r1_load_pair(phi, x, two);
                        if (!first) l[j] = r1_load_pair(D.lam, x, two);
                        r1_cost_pair<COST>(D.cost, x, two, c[j][0], c[j][1], ci[j][0], ci[j][1]);
                    }
                }
#pragma unroll
                for (int j = 0; j < kR1Pairs; j++) {
                    const int64_t x = xt + 2 * (threadIdx.x + j * kR1Threads);
                    if (x >= N) continue;
                    const bool two = x + 1 < N;
                    const float2 fo[2] = {make_float2(v[j].x, v[j].y), make_float2(v[j].z, v[j].w)};
                    const float2 lo[2] = {make_float2(l[j].x, l[j].y), make_float2(l[j].z, l[j].w)};
                    float2 nl[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    float2 np[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        if (e == 1 && !two) break;
                        const float C = c[j][e];
                        const float cs = C - c0;
                        float2 lv = first ? make_float2(cs * (fo[e].x + dl.x), cs * (fo[e].y + dl.y)) : lo[e];
                        lv.x += m.x;
                        lv.y += m.y;
                        s0 = fmaf(cs, fmaf(lv.x, fo[e].y, -lv.y * fo[e].x), s0);
                        if (round > 0) {
                            const float2 ph = r1_phase<COST>(stab, C, ci[j][e], cf);
                            nl[e] = r1_cmul_conj(lv, ph);  // mu e^{+i g C}
                            s1 += nl[e].x;
                            s2 += nl[e].y;
                            if (!D.ckpt) {
                                const float2 q = r1_cmul_conj(fo[e], ph);
                                np[e] = make_float2(q.x - dq.x, q.y - dq.y);
                            }
                        }
                    }
                    if (round > 0) {
                        if (two) {
                            r1_st2(D.lam + x, nl[0], nl[1]);
                            if (!D.ckpt) r1_st2(phi + x, np[0], np[1]);
                        } else {
                            D.lam[x] = nl[0];
                            if (!D.ckpt) phi[x] = np[0];
                        }
                    }
                }
            }
            acc[0] += (double)s0;
            acc[1] += (double)s1;
            acc[2] += (double)s2;
        }
        // t is now this block's first tile at or after t_end (the next unit's)
        r1_block_sum3(acc, red);
        if (threadIdx.x == 0) {
            double *pp = D.part + (size_t)slot * 3;
            pp[0] = acc[0];
            pp[1] = acc[1];
            pp[2] = acc[2];
        }
    }
}

// Scalars between passes, one block per unit: the unit's block slots summed
// in slot order, then the round's scalar formulas in float64.
//   R1_SFWD (round r): S_r = sum phi_r, d_r = (e^{-i b_r} - 1) S_r / N
//   R1_SLAST: <C> to E; with gradients c0 = <C>, sum lambda_{p-1} =
//             sum C psi - c0 sum psi, the beta_{p-1} partial and
//             m = (e^{+i b_{p-1}} - 1) sum lambda_{p-1} / N
//   R1_SBWD (round r): the gamma_r partial; for r > 0 the beta_{r-1} partial
//             and m for round r - 1
// Scalar layout per unit: [4 r + 0, 1] = d_r, [4 r + 2, 3] = S_r (r < p),
// [4 p] = c0, [4 p + 1, 2] = m of the round the adjoint is at.
__global__ void __launch_bounds__(kR1Threads) r1_scalar_kernel(const R1Desc *__restrict__ descs,
                                                              const uint32_t *__restrict__ tb, uint32_t grid,
                                                              int mode, int round) {
    __shared__ double red[3][kR1Threads / 32];
    const R1Desc D = descs[blockIdx.x];
    const uint32_t nt = tb[blockIdx.x + 1] - tb[blockIdx.x];
    const uint32_t ns = nt < grid ? nt : grid;
    double v[3] = {0.0, 0.0, 0.0};
    for (uint32_t i = threadIdx.x; i < ns; i += kR1Threads) {
        v[0] += D.part[3 * i];
        v[1] += D.part[3 * i + 1];
        v[2] += D.part[3 * i + 2];
    }
    r1_block_sum3(v, red);
    if (threadIdx.x != 0) return;
    const double A = v[0], B = v[1], Cs = v[2];
    double *sc = D.scal;
    const double N = (double)D.dim;
    const int p = D.p;
    constexpr double kInv2Pi = 0.15915494309189533577;
    // e^{s i b} - 1 = 2 i s sin(b/2) e^{s i b/2}: (re, im) without cancellation at small b
    auto mixer_factor = [&](double beta, double sgn, double &re, double &im) {
        double sh, ch;
        sincospi(beta * kInv2Pi, &sh, &ch);  // sin(b/2), cos(b/2)
        re = -2.0 * sh * sh;
        im = sgn * 2.0 * sh * ch;
    };
    if (mode == R1_SFWD) {
        double fr, fi;
        mixer_factor(D.angles[round], -1.0, fr, fi);
        sc[4 * round + 2] = A;
        sc[4 * round + 3] = B;
        sc[4 * round] = (fr * A - fi * B) / N;
        sc[4 * round + 1] = (fr * B + fi * A) / N;
        return;
    }
    // beta_r partial and m for round r from L = sum lambda_r
    auto adjoint_round = [&](int r, double Lr, double Li) {
        const double Pr = sc[4 * r + 2] + N * sc[4 * r];  // sum psi_r = S_r + N d_r
        const double Pi = sc[4 * r + 3] + N * sc[4 * r + 1];
        D.grad[r] = 2.0 * (Lr * Pi - Li * Pr) / N;
        double fr, fi;
        mixer_factor(D.angles[r], 1.0, fr, fi);
        sc[4 * p + 1] = (fr * Lr - fi * Li) / N;
        sc[4 * p + 2] = (fr * Li + fi * Lr) / N;
    };
    if (mode == R1_SLAST) {
        *D.E = A;
        if (!D.grad) return;
        sc[4 * p] = A;
        const double Pr = sc[4 * (p - 1) + 2] + N * sc[4 * (p - 1)];
        const double Pi = sc[4 * (p - 1) + 3] + N * sc[4 * (p - 1) + 1];
        adjoint_round(p - 1, B - A * Pr, Cs - A * Pi);
        return;
    }
    D.grad[p + round] = 2.0 * A;
    if (round > 0) adjoint_round(round - 1, B, Cs);
}

}  // namespace

int r1_tile_amps() { return kR1Tile; }

uint32_t r1_max_grid() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (uint32_t)std::max(1, nsm) * kR1BlocksPerSM;
}

uint32_t r1_grid(int mode, int cost_dtype) {
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const void *k;
    if (cost_dtype == 0)
        k = mode == R1_FWD ? (const void *)r1_pass_kernel<R1_FWD, 0>
                           : (mode == R1_LAST ? (const void *)r1_pass_kernel<R1_LAST, 0>
                                              : (const void *)r1_pass_kernel<R1_BWD, 0>);
    else
        k = mode == R1_FWD ? (const void *)r1_pass_kernel<R1_FWD, 1>
                           : (mode == R1_LAST ? (const void *)r1_pass_kernel<R1_LAST, 1>
                                              : (const void *)r1_pass_kernel<R1_BWD, 1>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kR1Threads, 0) != cudaSuccess || occ < 1) occ = 1;
    occ = std::min(occ, kR1BlocksPerSM);
    return (uint32_t)std::max(1, nsm) * (uint32_t)occ;
}

cudaError_t launch_r1_pass(int mode, int cost_dtype, const R1Desc *d, const uint32_t *tb, int nd, uint32_t tiles,
                           uint32_t grid, int round, cudaStream_t s) {
    if (tiles == 0 || grid == 0) return cudaSuccess;
    auto go = [&](auto kern) {
        kern<<<grid, kR1Threads, 0, s>>>(d, tb, nd, tiles, round);
        return cudaGetLastError();
    };
    if (cost_dtype == 0) {
        if (mode == R1_FWD) return go(r1_pass_kernel<R1_FWD, 0>);
        if (mode == R1_LAST) return go(r1_pass_kernel<R1_LAST, 0>);
        return go(r1_pass_kernel<R1_BWD, 0>);
    }
    if (mode == R1_FWD) return go(r1_pass_kernel<R1_FWD, 1>);
    if (mode == R1_LAST) return go(r1_pass_kernel<R1_LAST, 1>);
    return go(r1_pass_kernel<R1_BWD, 1>);
}

cudaError_t launch_r1_scalar(int mode, const R1Desc *d, const uint32_t *tb, int nd, uint32_t grid, int round,
                             cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    r1_scalar_kernel<<<nd, kR1Threads, 0, s>>>(d, tb, grid, mode, round);
    return cudaGetLastError();
}

}  // namespace qg
