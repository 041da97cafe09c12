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
// Data movement: a pass streams each vector once.  One producer warp per
// block copies whole tiles (2048 amplitudes, 16 KiB a vector, plus their cost
// values) into a ring of shared-memory stages with one-dimensional bulk (TMA)
// copies, completing on mbarriers; eight consumer warps compute from the
// stages and store results straight to global memory.  The ring keeps
// 130-200 KiB of loads in flight per SM whatever the consumers are doing.  A
// unit's last tile, when partial, is read by the consumers directly (a bulk
// copy needs a multiple of 16 bytes and must not read past a buffer).
//
// Sums: float32 over a thread's 8 amplitudes of a tile; across the tiles a
// thread visits in a compensated (Kahan) float32 pair, which keeps about
// float64 accuracy without float64 arithmetic per tile (slow on this part);
// float64 across the block and over the blocks, in a fixed order, so results
// are bitwise reproducible run to run.
#include "common.cuh"
#include "bulk.cuh"

#include <algorithm>
#include <cstdlib>

namespace qg {
namespace {

constexpr int kR1Threads = 256;                  // consumer threads (8 warps)
constexpr int kR1Block = kR1Threads + 32;        // + the producer warp
constexpr int kR1Pairs = 4;                      // amplitude pairs per consumer thread per tile
constexpr int kR1Tile = kR1Threads * kR1Pairs * 2;
constexpr uint32_t kR1VecB = kR1Tile * 8;        // one vector's tile, bytes
constexpr int kR1MaxStages = 16;
constexpr int kR1BlocksPerSM = 8;                // upper bound used to size the partial slots
// shared-memory head: full / empty barriers at 0, block-sum scratch at
// kR1RedOff, the phase table at kR1TabOff; the stages follow at kR1HeadB
constexpr uint32_t kR1RedOff = 2 * kR1MaxStages * 8;
constexpr uint32_t kR1TabOff = 512;
constexpr uint32_t kR1HeadB = kR1TabOff + kPhaseTable * 8;
static_assert(kR1RedOff + 3 * (kR1Threads / 32) * 8 <= kR1TabOff, "head layout");
static_assert(kR1HeadB % 128 == 0, "stage area alignment");
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

// Barrier over the kR1Threads consumer threads only (named barrier 1; the
// producer warp never takes part).
__device__ __forceinline__ void r1_consumer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kR1Threads) : "memory");
}

// Sum of three float64 values over the kR1Threads consumer threads (or the
// whole block of the scalar kernel, CONSUMERS false), in a fixed order; the
// result is valid in thread 0.  Every participating thread must call it.
template <bool CONSUMERS>
__device__ __forceinline__ void r1_block_sum3(double (&v)[3], double (*red)[kR1Threads / 32]) {
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (CONSUMERS) r1_consumer_sync();  // red is free (an earlier sum has been read)
    else __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 3; q++) red[q][w] = v[q];
    if (CONSUMERS) r1_consumer_sync();
    else __syncthreads();
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

// Compensated float32 running sum: the value is hi - lo.
struct Kahan {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - lo;
        const float t = hi + y;
        lo = (t - hi) - y;
        hi = t;
    }
    __device__ __forceinline__ double value() const { return (double)hi - (double)lo; }
};

template <int COST>
__device__ __forceinline__ float2 r1_phase(const float2 *stab, float C, int ci, const RoundCoef &cf) {
    if constexpr (COST == 1) return stab[ci];
    else return r1_phase_f32(C, cf.g_hi, cf.g_lo);
}

__device__ __forceinline__ void r1_st2(float2 *p, float2 a, float2 b) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a.x, a.y, b.x, b.y));
}
// Amplitude pair at even x (x + 1 < N), or the single amplitude x (global).
__device__ __forceinline__ float4 r1_load_pair(const float2 *p, int64_t x, bool two) {
    if (two) return __ldcs(reinterpret_cast<const float4 *>(p + x));
    const float2 a = p[x];
    return make_float4(a.x, a.y, 0.f, 0.f);
}

// Bytes of one stage: the tile of each vector the pass reads, then its costs.
template <int MODE, int COST>
struct R1Stage {
    static constexpr uint32_t kCostB = kR1Tile * (COST == 0 ? 4 : 1);
    static constexpr uint32_t kVecs = MODE == R1_BWD ? 2 : 1;  // phi (and lambda)
    static constexpr uint32_t kBytes = kVecs * kR1VecB + kCostB;
    static_assert(kBytes % 128 == 0, "stage alignment");
};

// Per-unit values the consumers need, read once when a block enters a unit.
struct R1Unit {
    const float2 *in;  // FWD: phi_{r-1} or the initial state; LAST / BWD: phi
    float2 *out;       // FWD: phi_r; BWD: phi_{r-1} (no checkpoints)
    int64_t N;
    uint32_t t_lo, t_hi, slot;
    float2 dp, dq, m;  // pending mixer shifts and the adjoint's m (see the modes)
    float c0;
    bool gen, first, ckpt;
};

// One streaming pass over every tile of every unit of the launch.  Tiles go to
// blocks round-robin (block b: tiles b, b + G, ...), so each unit's tiles form
// one run per block.  Modes, for round r:
//   R1_FWD : phi_r = (phi_{r-1} + d_{r-1}) e^{-i g_r C} (r = 0: the initial
//            state); sums (Re, Im) of phi_r
//   R1_LAST: psi = phi_{p-1} + d_{p-1}; sums C |psi|^2, Re and Im of C psi
//   R1_BWD : lambda_r (stored, or (C - c0) psi_{p-1} for r = p - 1), mu,
//            the gamma_r sum; for r > 0 lambda_{r-1} stored and summed, and
//            without checkpoints phi_{r-1} recovered in place
// Each block writes one (sum, sum, sum) slot per unit it visited: slot
// (b - tile_begin[unit]) mod G.
template <int MODE, int COST>
__global__ void __launch_bounds__(kR1Block, 1) r1_pass_kernel(const R1Desc *__restrict__ descs,
                                                              const uint32_t *__restrict__ tb, int nd,
                                                              uint32_t total, int round, int nst, int *err) {
    using SG = R1Stage<MODE, COST>;
    extern __shared__ __align__(128) unsigned char r1_smem[];
    uint64_t *full_bar = reinterpret_cast<uint64_t *>(r1_smem);
    uint64_t *empty_bar = full_bar + kR1MaxStages;
    double(*red)[kR1Threads / 32] = reinterpret_cast<double(*)[kR1Threads / 32]>(r1_smem + kR1RedOff);
    float2 *stab = reinterpret_cast<float2 *>(r1_smem + kR1TabOff);
    unsigned char *stages = r1_smem + kR1HeadB;
    const uint32_t G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int k = 0; k < nst; k++) {
            mbar_init(smem_u32(&full_bar[k]), 1);
            mbar_init(smem_u32(&empty_bar[k]), kR1Threads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kR1Threads / 32) {  // ---------------------------- producer
        if (lane != 0) return;
        bool fail = false;
        uint32_t t_hi = 0, t_lo = 0;
        int64_t N = 0;
        const void *src_v = nullptr, *src_l = nullptr, *src_c = nullptr;
        uint32_t i = 0;
        for (uint32_t t = blockIdx.x; t < total; t += G, i++) {
            const uint32_t s = i % (uint32_t)nst;
            const uint32_t fb = smem_u32(&full_bar[s]);
            if (i >= (uint32_t)nst && !fail && !mbar_wait(smem_u32(&empty_bar[s]), ((i / nst) - 1) & 1u)) {
                fail = true;
                atomicOr(err, DERR_TIMEOUT);
            }
            if (t >= t_hi) {
                const int di = r1_find(tb, nd, t);
                const R1Desc &D = descs[di];
                t_lo = tb[di];
                t_hi = tb[di + 1];
                N = D.dim;
                const int64_t ld = D.ld;
                src_c = D.cost;
                src_l = nullptr;
                if (MODE == R1_FWD)
                    src_v = round == 0 ? (const void *)D.init : (const void *)(D.phi + (D.ckpt ? (round - 1) * ld : 0));
                else if (MODE == R1_LAST)
                    src_v = D.phi + (D.ckpt ? (int64_t)(D.p - 1) * ld : 0);
                else {
                    src_v = D.phi + (D.ckpt ? (int64_t)round * ld : 0);
                    if (round != D.p - 1) src_l = D.lam;
                }
            }
            const int64_t x0 = (int64_t)(t - t_lo) * kR1Tile;
            if (fail || x0 + kR1Tile > N) {  // partial tile: the consumers read it themselves
                mbar_arrive_tx(fb, 0);
                continue;
            }
            const uint32_t bytes = (src_v ? kR1VecB : 0) + (src_l ? kR1VecB : 0) + SG::kCostB;
            mbar_arrive_tx(fb, bytes);
            const uint32_t sa = smem_u32(stages + (size_t)s * SG::kBytes);
            if (src_v) bulk_g2s(sa, static_cast<const float2 *>(src_v) + x0, kR1VecB, fb);
            if (src_l) bulk_g2s(sa + kR1VecB, static_cast<const float2 *>(src_l) + x0, kR1VecB, fb);
            bulk_g2s(sa + SG::kVecs * kR1VecB, static_cast<const unsigned char *>(src_c) + x0 * (COST == 0 ? 4 : 1),
                     SG::kCostB, fb);
        }
        return;
    }

    // ------------------------------------------------------------ consumers
    const int tid = threadIdx.x;
    R1Unit U{};
    const R1Desc *D = nullptr;
    RoundCoef cf{};
    Kahan acc[3];
    bool fail = false;
    auto flush = [&]() {
        double v[3] = {acc[0].value(), acc[1].value(), acc[2].value()};
        r1_block_sum3<true>(v, red);
        if (tid == 0) {
            double *pp = D->part + (size_t)U.slot * 3;
            pp[0] = v[0];
            pp[1] = v[1];
            pp[2] = v[2];
        }
        acc[0] = acc[1] = acc[2] = Kahan();
    };
    uint32_t i = 0;
    for (uint32_t t = blockIdx.x; t < total; t += G, i++) {
        const uint32_t s = i % (uint32_t)nst;
        if (!D || t >= U.t_hi) {  // entering a unit (uniform over the consumers)
            if (D) flush();
            const int di = r1_find(tb, nd, t);
            D = descs + di;
            U.t_lo = tb[di];
            U.t_hi = tb[di + 1];
            U.slot = (blockIdx.x + G - U.t_lo % G) % G;
            U.N = D->dim;
            const int64_t ld = D->ld;
            const int p = D->p;
            const double *sc = D->scal;
            cf = D->coef[round];
            U.ckpt = D->ckpt != 0;
            U.gen = MODE == R1_FWD && round == 0 && !D->init;
            U.first = MODE == R1_BWD && round == p - 1;
            if (MODE == R1_FWD) {
                U.in = round == 0 ? D->init : D->phi + (U.ckpt ? (int64_t)(round - 1) * ld : 0);
                U.out = D->phi + (U.ckpt ? (int64_t)round * ld : 0);
                U.dp = round == 0 ? make_float2(0.f, 0.f)
                                  : make_float2((float)sc[4 * (round - 1)], (float)sc[4 * (round - 1) + 1]);
            } else if (MODE == R1_LAST) {
                U.in = D->phi + (U.ckpt ? (int64_t)(p - 1) * ld : 0);
                U.dp = make_float2((float)sc[4 * (p - 1)], (float)sc[4 * (p - 1) + 1]);
            } else {
                U.out = D->phi + (U.ckpt ? (int64_t)round * ld : 0);
                U.in = U.out;
                U.c0 = (float)sc[4 * p];
                U.m = make_float2((float)sc[4 * p + 1], (float)sc[4 * p + 2]);
                U.dp = make_float2((float)sc[4 * round], (float)sc[4 * round + 1]);
                U.dq = round > 0 ? make_float2((float)sc[4 * (round - 1)], (float)sc[4 * (round - 1) + 1])
                                 : make_float2(0.f, 0.f);
            }
            if (COST == 1 && MODE != R1_LAST) {
                r1_consumer_sync();  // the previous unit's table is no longer read
                for (int k = tid; k < kPhaseTable; k += kR1Threads) stab[k] = D->table[round * kPhaseTable + k];
                r1_consumer_sync();
            }
        }
        bool ok = !fail && mbar_wait(smem_u32(&full_bar[s]), (i / nst) & 1u);
        if (!ok && !fail) {
            fail = true;
            atomicOr(err, DERR_TIMEOUT);
        }
        if (!fail) {
            const int64_t N = U.N;
            const int64_t xt = (int64_t)(t - U.t_lo) * kR1Tile;
            const bool staged = xt + kR1Tile <= N;
            const unsigned char *sb = stages + (size_t)s * SG::kBytes;
            const float4 *sv = reinterpret_cast<const float4 *>(sb);
            const float4 *sl = reinterpret_cast<const float4 *>(sb + kR1VecB);
            const unsigned char *scb = sb + SG::kVecs * kR1VecB;
            float4 v[kR1Pairs], l[kR1Pairs];
            float c[kR1Pairs][2];
            int ci[kR1Pairs][2];
            // ---- loads: from the stage, or (partial tile) from global memory
#pragma unroll
            for (int j = 0; j < kR1Pairs; j++) {
                const int q = tid + j * kR1Threads;  // pair index within the tile
                const int64_t x = xt + 2 * q;
                v[j] = U.gen ? make_float4(D->amp0, 0.f, D->amp0, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
                l[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                c[j][0] = c[j][1] = 0.f;
                ci[j][0] = ci[j][1] = 0;
                if (staged) {
                    if (!U.gen) v[j] = sv[q];
                    if (MODE == R1_BWD && !U.first) l[j] = sl[q];
                    if (COST == 0) {
                        const float2 cc = reinterpret_cast<const float2 *>(scb)[q];
                        c[j][0] = cc.x;
                        c[j][1] = cc.y;
                    } else {
                        const uchar2 cc = reinterpret_cast<const uchar2 *>(scb)[q];
                        ci[j][0] = cc.x;
                        ci[j][1] = cc.y;
                        c[j][0] = (float)cc.x;
                        c[j][1] = (float)cc.y;
                    }
                } else if (x < N) {
                    const bool two = x + 1 < N;
                    if (!U.gen) v[j] = r1_load_pair(U.in, x, two);
                    if (MODE == R1_BWD && !U.first) l[j] = r1_load_pair(D->lam, x, two);
                    r1_cost_pair<COST>(D->cost, x, two, c[j][0], c[j][1], ci[j][0], ci[j][1]);
                }
            }
            // ---- arithmetic and stores
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < kR1Pairs; j++) {
                const int64_t x = xt + 2 * (tid + j * kR1Threads);
                if (x >= N) continue;
                const bool two = x + 1 < N;
                const float2 fo[2] = {make_float2(v[j].x, v[j].y), make_float2(v[j].z, v[j].w)};
                if constexpr (MODE == R1_FWD) {
                    float2 a[2];
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        a[e] = r1_cmul(make_float2(fo[e].x + U.dp.x, fo[e].y + U.dp.y),
                                       r1_phase<COST>(stab, c[j][e], ci[j][e], cf));
                        if (e == 0 || two) {
                            s0 += a[e].x;
                            s1 += a[e].y;
                        }
                    }
                    if (two) r1_st2(U.out + x, a[0], a[1]);
                    else U.out[x] = a[0];
                } else if constexpr (MODE == R1_LAST) {
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        if (e == 1 && !two) break;
                        const float re = fo[e].x + U.dp.x, im = fo[e].y + U.dp.y, C = c[j][e];
                        s0 = fmaf(C, fmaf(re, re, im * im), s0);
                        s1 = fmaf(C, re, s1);
                        s2 = fmaf(C, im, s2);
                    }
                } else {
                    const float2 lo[2] = {make_float2(l[j].x, l[j].y), make_float2(l[j].z, l[j].w)};
                    float2 nl[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    float2 np[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        if (e == 1 && !two) break;
                        const float C = c[j][e];
                        const float cs = C - U.c0;
                        float2 lv = U.first ? make_float2(cs * (fo[e].x + U.dp.x), cs * (fo[e].y + U.dp.y)) : lo[e];
                        lv.x += U.m.x;
                        lv.y += U.m.y;
                        s0 = fmaf(cs, fmaf(lv.x, fo[e].y, -lv.y * fo[e].x), s0);  // (C - c0) Im(conj(mu) phi)
                        if (round > 0) {
                            const float2 ph = r1_phase<COST>(stab, C, ci[j][e], cf);
                            nl[e] = r1_cmul_conj(lv, ph);  // mu e^{+i g C}
                            s1 += nl[e].x;
                            s2 += nl[e].y;
                            if (!U.ckpt) {
                                const float2 q = r1_cmul_conj(fo[e], ph);
                                np[e] = make_float2(q.x - U.dq.x, q.y - U.dq.y);
                            }
                        }
                    }
                    if (round > 0) {
                        if (two) {
                            r1_st2(D->lam + x, nl[0], nl[1]);
                            if (!U.ckpt) r1_st2(U.out + x, np[0], np[1]);
                        } else {
                            D->lam[x] = nl[0];
                            if (!U.ckpt) U.out[x] = np[0];
                        }
                    }
                }
            }
            acc[0].add(s0);
            acc[1].add(s1);
            if (MODE != R1_FWD) acc[2].add(s2);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty_bar[s]));  // this warp is done with stage s
    }
    if (D) flush();
    if (fail && tid == 0)  // let copies still in flight land before the block exits
        for (int k = 0; k < nst; k++) mbar_wait(smem_u32(&full_bar[k]), 0u), mbar_wait(smem_u32(&full_bar[k]), 1u);
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
    r1_block_sum3<false>(v, red);
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

// Stages per block and blocks per SM of one pass kernel (loads in flight per
// SM: stages x blocks x stage bytes, at most about 200 KiB of the SM's shared
// memory).  Defaults, measured at 2^28 amplitudes: 4 stages with uint8
// costs, 3 with float32 (about 72 KiB of forward loads in flight per SM; a
// deeper ring lost 5-10%, reads running far ahead of the stream of writes);
// one block per SM for the forward and adjoint passes, two for the read-only
// <C> pass, whose 16 consumer warps keep up with the loads where 8 did not
// (uint8 costs: 6.8 TB/s against 4.7).  QAOA_R1_STAGES / QAOA_R1_BLOCKS
// override.
struct R1Config {
    int nst, bps;
    uint32_t smem;
};
template <int MODE, int COST>
R1Config r1_config() {
    using SG = R1Stage<MODE, COST>;
    const char *e1 = getenv("QAOA_R1_STAGES");
    const char *e2 = getenv("QAOA_R1_BLOCKS");
    int bps = e2 ? atoi(e2) : (MODE == R1_LAST ? 2 : 1);
    bps = std::max(1, std::min(bps, 4));
    const int room = (int)((200u * 1024u) / (uint32_t)bps) - (int)kR1HeadB;
    int nst = e1 ? atoi(e1) : (COST == 1 ? 4 : 3);
    nst = std::max(2, std::min(nst, std::min(kR1MaxStages, room / (int)SG::kBytes)));
    return {nst, bps, kR1HeadB + (uint32_t)nst * SG::kBytes};
}

int r1_tile_amps() { return kR1Tile; }

uint32_t r1_max_grid() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (uint32_t)std::max(1, nsm) * kR1BlocksPerSM;
}

uint32_t r1_grid(int mode, int cost_dtype) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    R1Config c;
    if (cost_dtype == 0)
        c = mode == R1_FWD ? r1_config<R1_FWD, 0>() : (mode == R1_LAST ? r1_config<R1_LAST, 0>() : r1_config<R1_BWD, 0>());
    else
        c = mode == R1_FWD ? r1_config<R1_FWD, 1>() : (mode == R1_LAST ? r1_config<R1_LAST, 1>() : r1_config<R1_BWD, 1>());
    return (uint32_t)std::max(1, nsm) * (uint32_t)std::min(c.bps, kR1BlocksPerSM);
}

template <int MODE, int COST>
cudaError_t r1_go(const R1Desc *d, const uint32_t *tb, int nd, uint32_t tiles, uint32_t grid, int round, int *err,
                  cudaStream_t s) {
    static int attr_done[kMaxDevices] = {0};
    const R1Config c = r1_config<MODE, COST>();
    cudaError_t e = smem_attr_once(r1_pass_kernel<MODE, COST>, (int)c.smem, attr_done);
    if (e != cudaSuccess) return e;
    r1_pass_kernel<MODE, COST><<<grid, kR1Block, c.smem, s>>>(d, tb, nd, tiles, round, c.nst, err);
    return cudaGetLastError();
}

cudaError_t launch_r1_pass(int mode, int cost_dtype, const R1Desc *d, const uint32_t *tb, int nd, uint32_t tiles,
                           uint32_t grid, int round, int *err, cudaStream_t s) {
    if (tiles == 0 || grid == 0) return cudaSuccess;
    if (cost_dtype == 0) {
        if (mode == R1_FWD) return r1_go<R1_FWD, 0>(d, tb, nd, tiles, grid, round, err, s);
        if (mode == R1_LAST) return r1_go<R1_LAST, 0>(d, tb, nd, tiles, grid, round, err, s);
        return r1_go<R1_BWD, 0>(d, tb, nd, tiles, grid, round, err, s);
    }
    if (mode == R1_FWD) return r1_go<R1_FWD, 1>(d, tb, nd, tiles, grid, round, err, s);
    if (mode == R1_LAST) return r1_go<R1_LAST, 1>(d, tb, nd, tiles, grid, round, err, s);
    return r1_go<R1_BWD, 1>(d, tb, nd, tiles, grid, round, err, s);
}

cudaError_t launch_r1_scalar(int mode, const R1Desc *d, const uint32_t *tb, int nd, uint32_t grid, int round,
                             cudaStream_t s) {
    if (nd <= 0) return cudaSuccess;
    r1_scalar_kernel<<<nd, kR1Threads, 0, s>>>(d, tb, grid, mode, round);
    return cudaGetLastError();
}

}  // namespace qg
