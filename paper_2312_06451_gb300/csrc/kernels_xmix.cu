// Transverse-field (X) mixer path: phase separator, per-qubit mixer
// rotations, expectation and adjoint (reverse-mode) gradient on complex64
// states.
//
// Method (arXiv 2312.06451): round k applies e^{-i gamma_k C} elementwise and
// then e^{-i beta_k sum_i X_i} (Eq. 1).  Because the X_i commute, the mixer is
// n independent single-qubit rotations (Sec. 2.2; Eq. 2 is the equivalent
// Hadamard-diagonal form), each mixing the amplitude pairs (x, x xor 2^i).
//
// Kernel design (sm_103a, HBM-bound):
//   * A pass streams the state once through the SMs in tiles of 2^T
//     amplitudes and applies every rotation whose qubit is a tile bit, so one
//     round costs ceil(n / T)-ish passes instead of n sweeps.  The first pass
//     of a tile set covers qubits 0..T-1 with fully contiguous tiles; later
//     passes gather 2^c contiguous amplitudes (c >= 4: whole 128-byte lines)
//     times 2^(T-c) strided ones to reach the high qubits.
//   * Each thread holds 32 amplitudes in registers.  A tile goes through three
//     register layouts ("stages"): the first is the coalesced 16-byte load
//     layout, the third the coalesced store layout; two shared-memory
//     transposes (XOR-swizzled, bank-conflict free) move between them.  Every
//     rotation happens in registers, on the stage where its bit is a register
//     bit.
//   * The phase e^{-i gamma C} is applied as the tile is loaded, the
//     expectation sum |psi|^2 C as it is stored, so neither costs a pass.
//   * The adjoint pass carries lambda and psi together, undoing the rotations
//     of both and accumulating 2 Im <lambda|X_i|psi> for the beta derivative
//     as each qubit comes by (valid at any point of the round because all
//     X_i commute); the gamma derivative 2 Im <mu|C|phi> and the undone phase
//     are fused into the last adjoint pass of the round.
//   * Partial sums are per tile in float32, combined in float64 in a fixed
//     order, so results are bitwise reproducible.
#include "common.cuh"

#include <math.h>

namespace qg {
namespace {

constexpr float kTwoPiF = 6.2831853071795864769f;
constexpr double kTwoPi = 6.2831853071795864769;

// XOR swizzle of a tile-local amplitude index into shared memory.  Bits 1..3
// are flipped by a fold of bits 6..14, bit 0 is kept so that the amplitude
// pair (l, l^1) stays one aligned 16-byte vector.  With it, every stage's
// accesses are conflict free: 16-byte accesses vary local bits 1..3 within a
// quarter warp; 8-byte accesses vary local bits {0,6,7,8} (stage 2) or
// {0,1,2,3} (stage 3) within a half warp.  The map is linear over GF(2):
// swz(a ^ b) = swz(a) ^ swz(b).
__device__ __forceinline__ uint32_t swz(uint32_t l) {
    return l ^ ((((l >> 6) ^ (l >> 9) ^ (l >> 12)) & 7u) << 1);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// e^{-i gamma C} for a float32 cost.  gamma/(2 pi) = g_hi + g_lo; the product
// t = (g_hi + g_lo) C is formed as a float pair (exact head product by FMA),
// its integer part removed exactly, and the remaining turn f in [-1/2, 1/2]
// fed to the hardware sine/cosine at 2 pi f in [-pi, pi].
__device__ __forceinline__ float2 phase_f32(float C, float ghi, float glo) {
    const float th = ghi * C;
    const float te = fmaf(ghi, C, -th);
    const float tl = fmaf(glo, C, te);
    const float f = (th - rintf(th)) + tl;
    float s, c;
    __sincosf(kTwoPiF * f, &s, &c);
    return make_float2(c, -s);
}

// Rotation e^{-i b X} on register pairs (i, i | 1<<RB), without its scalar
// factor (see RoundCoef).
template <int RB>
__device__ __forceinline__ void rot_pairs(float2 (&a)[32], float t, int mode) {
    if (mode == 0) {
#pragma unroll
        for (int i = 0; i < 32; i++) {
            if (i & (1 << RB)) continue;
            const int j = i | (1 << RB);
            const float2 x = a[i], y = a[j];
            a[i] = make_float2(fmaf(t, y.y, x.x), fmaf(-t, y.x, x.y));
            a[j] = make_float2(fmaf(t, x.y, y.x), fmaf(-t, x.x, y.y));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; i++) {
            if (i & (1 << RB)) continue;
            const int j = i | (1 << RB);
            const float2 x = a[i], y = a[j];
            a[i] = make_float2(fmaf(t, x.x, y.y), fmaf(t, x.y, -y.x));
            a[j] = make_float2(fmaf(t, y.x, x.y), fmaf(t, y.y, -x.x));
        }
    }
}

// sum over register pairs of Im( conj(l_a) p_b + conj(l_b) p_a ), i.e. this
// thread's share of Im <l| X_q |p> for the qubit on register bit RB.
template <int RB>
__device__ __forceinline__ float pair_im(const float2 (&l)[32], const float2 (&p)[32]) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (i & (1 << RB)) continue;
        const int j = i | (1 << RB);
        s = fmaf(l[i].x, p[j].y, s);
        s = fmaf(-l[i].y, p[j].x, s);
        s = fmaf(l[j].x, p[i].y, s);
        s = fmaf(-l[j].y, p[i].x, s);
    }
    return s;
}

// One rotation step on register bit RB if its local qubit is active.
template <int RB, int BWD>
__device__ __forceinline__ void rot_step(float2 (&a)[32], float2 (&b)[32], uint32_t active, int lb,
                                         float t, int mode, float sc2, float &pscale, float &bacc) {
    if (!((active >> lb) & 1u)) return;
    if (BWD) {
        bacc = fmaf(pair_im<RB>(b, a), pscale, bacc);
        pscale *= sc2;
        rot_pairs<RB>(b, t, mode);
    }
    rot_pairs<RB>(a, t, mode);
}

// Deterministic block sum of one float per thread, accumulated in float64;
// the result is valid in thread 0.
template <int NW>
__device__ __forceinline__ double block_sum(float v, double *red) {
    double d = (double)v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = d;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NW; w++) tot += red[w];
    }
    __syncthreads();
    return tot;
}

__device__ __forceinline__ int find_desc(const uint32_t *__restrict__ tile_begin, int ndesc,
                                         uint32_t b) {
    int lo = 0, hi = ndesc - 1, found = -1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        if (tile_begin[mid] <= b) {
            found = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    if (found >= 0 && b >= tile_begin[found + 1]) found = -1;
    return found;
}

// --------------------------------------------------------------------------
// The pass kernel.  T: tile bits; BWD: 0 forward, 1 adjoint; COST: 0 float32,
// 1 uint8 cost.  Register layouts of a tile (local bit numbers), W = T - 10:
//   stage 1: amp bit 0 -> local 0 (inside a 16-byte vector), lanes -> 1..5,
//            warps -> 6..5+W, amp bits 1..4 -> 6+W..T-1
//   stage 2: amp bits 0..4 -> 1..5, lanes -> {0,6,7,8,9}, warps -> 10..T-1
//   stage 3: amp bits 0..4 -> 6..10, lanes -> 0..4, warps -> {5, 11..T-1}
// Rotated on stage 1: local 0 and 6+W..T-1; stage 2: 1..5; stage 3: 6..5+W.
template <int T, int BWD, int COST>
__global__ void __launch_bounds__(1 << (T - 5), (BWD || T >= 14) ? 1 : 2)
xpass_kernel(const PassDesc *__restrict__ descs, const uint32_t *__restrict__ tile_begin,
             int ndesc, int *err) {
    constexpr int NT = 1 << (T - 5);
    constexpr int NW = NT / 32;
    constexpr int W = T - 10;
    constexpr int S1R0 = 6 + W;
    constexpr int TILE = 1 << T;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sm_a = reinterpret_cast<float2 *>(smem_raw);
    float2 *sm_b = sm_a + TILE;                         // adjoint only
    float2 *stab = sm_a + (BWD ? 2 : 1) * TILE;          // phase table
    __shared__ PassDesc D;
    __shared__ int s_di;
    __shared__ double s_red[NW];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_di = find_desc(tile_begin, ndesc, blockIdx.x);
    __syncthreads();
    const int di = s_di;
    if (di < 0) {
        if (tid == 0) atomicOr(err, DERR_BAD_DESC);
        return;
    }
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + di);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&D);
        for (int i = tid; i < (int)(sizeof(PassDesc) / 4); i += NT) dst[i] = src[i];
    }
    __syncthreads();
    const uint32_t tile = blockIdx.x - tile_begin[di];
    const uint32_t flags = D.flags;
    const uint32_t active = D.active;

    if (COST == 1 && (flags & PF_PHASE)) {
        for (int i = tid; i < kPhaseTable; i += NT) stab[i] = D.table[i];
        __syncthreads();
    }

    const RoundCoef cf = *D.coef;
    float t = cf.bt, sc = cf.bs;
    const int mode = cf.bmode;
    if (BWD) {  // undo: e^{+i b X}, i.e. the coefficients of -b
        t = -t;
        if (mode) sc = -sc;
    }
    const float sc2 = sc * sc;
    const float ghi = cf.g_hi, glo = cf.g_lo;

    // Element offsets fit 32 bits: the X path is limited to n <= 32.
    uint32_t base = 0;
    for (int bb = 0; bb < D.nfree; bb++) base |= ((tile >> bb) & 1u) << D.fpos[bb];
    auto gofs = [&](uint32_t l) {
        uint32_t o = 0;
#pragma unroll
        for (int j = 0; j < T; j++)
            if ((l >> j) & 1u) o += 1u << D.gpos[j];
        return o;
    };

    float2 a[32];  // psi
    float2 b[32];  // lambda (adjoint)
    float pscale = 1.f, bacc = 0.f;

    // ---------------- stage 1: coalesced load, phase / lambda = C psi
    const uint32_t l1 = ((uint32_t)lane << 1) | ((uint32_t)warp << 6);
    {
        const uint32_t g1 = base + gofs(l1);
        uint32_t rs[4];
#pragma unroll
        for (int k = 0; k < 4; k++) rs[k] = 1u << D.gpos[S1R0 + k];
        const bool gen = !BWD && (flags & PF_GEN_INIT);
        const bool need_c = BWD ? (flags & PF_LAM_FROM_C) : (flags & PF_PHASE);
#pragma unroll
        for (int r = 0; r < 16; r++) {
            const uint32_t off = g1 + ((r & 1) ? rs[0] : 0) + ((r & 2) ? rs[1] : 0) +
                                 ((r & 4) ? rs[2] : 0) + ((r & 8) ? rs[3] : 0);
            if (gen) {
                a[2 * r] = make_float2(D.amp0, 0.f);
                a[2 * r + 1] = make_float2(D.amp0, 0.f);
            } else {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(D.psi_in + off));
                a[2 * r] = make_float2(v.x, v.y);
                a[2 * r + 1] = make_float2(v.z, v.w);
            }
            if (BWD && !(flags & PF_LAM_FROM_C)) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(D.lam_in + off));
                b[2 * r] = make_float2(v.x, v.y);
                b[2 * r + 1] = make_float2(v.z, v.w);
            }
            if (need_c) {
                float c0, c1;
                if (COST == 0) {
                    const float2 cc = __ldg(reinterpret_cast<const float2 *>(D.cost) + (off >> 1));
                    c0 = cc.x;
                    c1 = cc.y;
                } else {
                    const uchar2 cc = __ldg(reinterpret_cast<const uchar2 *>(D.cost) + (off >> 1));
                    c0 = (float)cc.x;
                    c1 = (float)cc.y;
                    if (!BWD) {
                        a[2 * r] = cmul(a[2 * r], stab[cc.x]);
                        a[2 * r + 1] = cmul(a[2 * r + 1], stab[cc.y]);
                    }
                }
                if (BWD) {
                    b[2 * r] = make_float2(c0 * a[2 * r].x, c0 * a[2 * r].y);
                    b[2 * r + 1] = make_float2(c1 * a[2 * r + 1].x, c1 * a[2 * r + 1].y);
                } else if (COST == 0) {
                    a[2 * r] = cmul(a[2 * r], phase_f32(c0, ghi, glo));
                    a[2 * r + 1] = cmul(a[2 * r + 1], phase_f32(c1, ghi, glo));
                }
            }
        }
    }
    rot_step<0, BWD>(a, b, active, 0, t, mode, sc2, pscale, bacc);
    rot_step<1, BWD>(a, b, active, S1R0 + 0, t, mode, sc2, pscale, bacc);
    rot_step<2, BWD>(a, b, active, S1R0 + 1, t, mode, sc2, pscale, bacc);
    rot_step<3, BWD>(a, b, active, S1R0 + 2, t, mode, sc2, pscale, bacc);
    rot_step<4, BWD>(a, b, active, S1R0 + 3, t, mode, sc2, pscale, bacc);

    // ---------------- stage 1 -> stage 2 transpose
    const uint32_t p1 = swz(l1);
#pragma unroll
    for (int r = 0; r < 16; r++) {
        const uint32_t idx = p1 ^ swz((uint32_t)r << S1R0);
        *reinterpret_cast<float4 *>(sm_a + idx) =
            make_float4(a[2 * r].x, a[2 * r].y, a[2 * r + 1].x, a[2 * r + 1].y);
        if (BWD)
            *reinterpret_cast<float4 *>(sm_b + idx) =
                make_float4(b[2 * r].x, b[2 * r].y, b[2 * r + 1].x, b[2 * r + 1].y);
    }
    __syncthreads();
    const uint32_t l2 = ((uint32_t)lane & 1u) | ((((uint32_t)lane >> 1) & 15u) << 6) |
                        ((uint32_t)warp << 10);
    const uint32_t p2 = swz(l2);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        a[i] = sm_a[p2 ^ swz((uint32_t)i << 1)];
        if (BWD) b[i] = sm_b[p2 ^ swz((uint32_t)i << 1)];
    }
    rot_step<0, BWD>(a, b, active, 1, t, mode, sc2, pscale, bacc);
    rot_step<1, BWD>(a, b, active, 2, t, mode, sc2, pscale, bacc);
    rot_step<2, BWD>(a, b, active, 3, t, mode, sc2, pscale, bacc);
    rot_step<3, BWD>(a, b, active, 4, t, mode, sc2, pscale, bacc);
    rot_step<4, BWD>(a, b, active, 5, t, mode, sc2, pscale, bacc);

    // ---------------- stage 2 -> stage 3 transpose
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i++) {
        sm_a[p2 ^ swz((uint32_t)i << 1)] = a[i];
        if (BWD) sm_b[p2 ^ swz((uint32_t)i << 1)] = b[i];
    }
    __syncthreads();
    const uint32_t l3 = (uint32_t)lane | (((uint32_t)warp & 1u) << 5) | (((uint32_t)warp >> 1) << 11);
    const uint32_t p3 = swz(l3);
#pragma unroll
    for (int i = 0; i < 32; i++) {
        a[i] = sm_a[p3 ^ swz((uint32_t)i << 6)];
        if (BWD) b[i] = sm_b[p3 ^ swz((uint32_t)i << 6)];
    }
    rot_step<0, BWD>(a, b, active, 6, t, mode, sc2, pscale, bacc);
    if (W > 1) rot_step<1, BWD>(a, b, active, 7, t, mode, sc2, pscale, bacc);
    if (W > 2) rot_step<2, BWD>(a, b, active, 8, t, mode, sc2, pscale, bacc);
    if (W > 3) rot_step<3, BWD>(a, b, active, 9, t, mode, sc2, pscale, bacc);

    // ---------------- stage 3: scalar factor, fused epilogue, coalesced store
    {
        float fs = 1.f;
        const int nrot = __popc(active);
        for (int k = 0; k < nrot; k++) fs *= sc;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            a[i].x *= fs;
            a[i].y *= fs;
            if (BWD) {
                b[i].x *= fs;
                b[i].y *= fs;
            }
        }
    }
    const uint32_t g3 = base + gofs(l3);
    uint32_t rs3[5];
#pragma unroll
    for (int k = 0; k < 5; k++) rs3[k] = 1u << D.gpos[6 + k];
    const bool epi_c = BWD ? (flags & PF_PHASE) : (flags & PF_E);
    float eacc = 0.f;
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const uint32_t off = g3 + ((i & 1) ? rs3[0] : 0) + ((i & 2) ? rs3[1] : 0) +
                             ((i & 4) ? rs3[2] : 0) + ((i & 8) ? rs3[3] : 0) +
                             ((i & 16) ? rs3[4] : 0);
        if (epi_c) {
            float C;
            float2 ph;
            if (COST == 0) {
                C = __ldg(reinterpret_cast<const float *>(D.cost) + off);
                if (BWD) ph = phase_f32(C, ghi, glo);
            } else {
                const unsigned char cc = __ldg(reinterpret_cast<const unsigned char *>(D.cost) + off);
                C = (float)cc;
                if (BWD) ph = stab[cc];
            }
            if (!BWD) {
                eacc = fmaf(C, fmaf(a[i].x, a[i].x, a[i].y * a[i].y), eacc);
            } else {
                // gamma partial: C Im(conj(mu) phi), then undo the phase
                eacc = fmaf(C, fmaf(b[i].x, a[i].y, -b[i].y * a[i].x), eacc);
                b[i] = cmul_conj(b[i], ph);
                if (flags & PF_UNPHASE_PSI) a[i] = cmul_conj(a[i], ph);
            }
        }
        if (D.psi_out) __stcs(D.psi_out + off, a[i]);
        if (BWD && D.lam_out) __stcs(D.lam_out + off, b[i]);
    }
    if (BWD) {
        const double tb = block_sum<NW>(bacc, s_red);
        if (tid == 0 && D.part_beta) D.part_beta[tile] = tb;
        if (flags & PF_PHASE) {
            const double tg = block_sum<NW>(eacc, s_red);
            if (tid == 0 && D.part_gamma) D.part_gamma[tile] = tg;
        }
    } else if (flags & PF_E) {
        const double te = block_sum<NW>(eacc, s_red);
        if (tid == 0 && D.part_E) D.part_E[tile] = te;
    }
}

// --------------------------------------------------------------------------
// Whole state in shared memory (n <= kSmallMaxN): all p rounds, the
// expectation and (GRAD) the adjoint sweep in one block per unit.  The adjoint
// undoes each round on psi in place.
constexpr int kSmallMaxN = 12;
constexpr int kSmallThreads = 256;

template <int COST, int GRAD>
__global__ void __launch_bounds__(kSmallThreads)
small_kernel(const SmallDesc *__restrict__ descs, int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[kSmallThreads / 32];
    const SmallDesc D = descs[blockIdx.x];
    const int N = 1 << D.n, H = N >> 1, n = D.n, p = D.p;
    float2 *psi = reinterpret_cast<float2 *>(smem_raw);
    float2 *lam = psi + N;
    float2 *tab = psi + 2 * N;
    const int tid = threadIdx.x;
    (void)err;

    auto costv = [&](int x) -> float {
        if (COST == 0) return __ldg(reinterpret_cast<const float *>(D.cost) + x);
        return (float)__ldg(reinterpret_cast<const unsigned char *>(D.cost) + x);
    };
    auto phase = [&](int x, const RoundCoef &cf) -> float2 {
        if (COST == 0) return phase_f32(costv(x), cf.g_hi, cf.g_lo);
        return tab[__ldg(reinterpret_cast<const unsigned char *>(D.cost) + x)];
    };
    auto load_table = [&](int k) {
        if (COST == 1) {
            __syncthreads();
            for (int i = tid; i < kPhaseTable; i += kSmallThreads)
                tab[i] = D.table[k * kPhaseTable + i];
            __syncthreads();
        }
    };
    // e^{-i b X_q} on every pair of qubit q (cb, sb: cos b, sin b)
    auto mix = [&](float2 *v, int q, float cb, float sb) {
        for (int j = tid; j < H; j += kSmallThreads) {
            const int lo = j & ((1 << q) - 1);
            const int x0 = ((j - lo) << 1) | lo, x1 = x0 | (1 << q);
            const float2 u = v[x0], w = v[x1];
            v[x0] = make_float2(fmaf(cb, u.x, sb * w.y), fmaf(cb, u.y, -sb * w.x));
            v[x1] = make_float2(fmaf(cb, w.x, sb * u.y), fmaf(cb, w.y, -sb * u.x));
        }
    };

    for (int x = tid; x < N; x += kSmallThreads)
        psi[x] = D.init ? D.init[x] : make_float2(D.amp0, 0.f);
    for (int k = 0; k < p; k++) {
        const RoundCoef cf = D.coef[k];
        __syncthreads();
        load_table(k);
        for (int x = tid; x < N; x += kSmallThreads) psi[x] = cmul(psi[x], phase(x, cf));
        for (int q = 0; q < n; q++) {
            __syncthreads();
            mix(psi, q, cf.cb, cf.sb);
        }
    }
    __syncthreads();
    float e = 0.f;
    for (int x = tid; x < N; x += kSmallThreads)
        e = fmaf(costv(x), fmaf(psi[x].x, psi[x].x, psi[x].y * psi[x].y), e);
    const double E = block_sum<kSmallThreads / 32>(e, s_red);
    if (tid == 0) *D.E_out = E;
    if constexpr (GRAD) {
    for (int x = tid; x < N; x += kSmallThreads) {
        const float c = costv(x);
        lam[x] = make_float2(c * psi[x].x, c * psi[x].y);
    }
    for (int k = p - 1; k >= 0; k--) {
        const RoundCoef cf = D.coef[k];
        __syncthreads();
        float gb = 0.f;
        for (int q = 0; q < n; q++) {
            for (int j = tid; j < H; j += kSmallThreads) {
                const int lo = j & ((1 << q) - 1);
                const int x0 = ((j - lo) << 1) | lo, x1 = x0 | (1 << q);
                const float2 l0 = lam[x0], l1 = lam[x1], a0 = psi[x0], a1 = psi[x1];
                gb += l0.x * a1.y - l0.y * a1.x + l1.x * a0.y - l1.y * a0.x;
            }
        }
        const double GB = block_sum<kSmallThreads / 32>(gb, s_red);
        if (tid == 0) D.grad_out[k] = 2.0 * GB;
        for (int q = 0; q < n; q++) {
            __syncthreads();
            mix(lam, q, cf.cb, -cf.sb);
            mix(psi, q, cf.cb, -cf.sb);
        }
        __syncthreads();
        load_table(k);
        float gg = 0.f;
        for (int x = tid; x < N; x += kSmallThreads) {
            const float2 l = lam[x], a = psi[x];
            gg = fmaf(costv(x), l.x * a.y - l.y * a.x, gg);
        }
        const double GG = block_sum<kSmallThreads / 32>(gg, s_red);
        if (tid == 0) D.grad_out[p + k] = 2.0 * GG;
        for (int x = tid; x < N; x += kSmallThreads) {
            const float2 ph = phase(x, cf);
            lam[x] = cmul_conj(lam[x], ph);
            psi[x] = cmul_conj(psi[x], ph);
        }
    }
    }  // GRAD
}

// --------------------------------------------------------------------------
// Angles -> per-round coefficients and uint8 phase tables (float64 math).
__global__ void __launch_bounds__(256) prep_kernel(const PrepDesc *__restrict__ descs, int *err) {
    const PrepDesc D = descs[blockIdx.x];
    for (int k = threadIdx.x; k < D.p; k += blockDim.x) {
        const double be = D.angles[k], ga = D.angles[D.p + k];
        if (!isfinite(be) || !isfinite(ga)) atomicOr(err, DERR_BAD_ANGLE);
        const double cb = cos(be), sb = sin(be);
        RoundCoef c;
        if (fabs(cb) >= fabs(sb)) {
            c.bmode = 0;
            c.bt = (float)(sb / cb);
            c.bs = (float)cb;
        } else {
            c.bmode = 1;
            c.bt = (float)(cb / sb);
            c.bs = (float)sb;
        }
        const double g = ga / kTwoPi;
        c.g_hi = (float)g;
        c.g_lo = (float)(g - (double)c.g_hi);
        c.cb = (float)cb;
        c.sb = (float)sb;
        c.pad = 0.f;
        D.coef[k] = c;
    }
    if (D.table) {
        const int tot = D.p * D.tsize;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int k = e / D.tsize, cst = e - k * D.tsize;
            double s, c;
            sincos(D.angles[D.p + k] * (double)cst, &s, &c);
            D.table[k * kPhaseTable + cst] = make_float2((float)c, (float)(-s));
        }
    }
}

// Fixed-order reduction of the per-tile partials of every unit.
__global__ void __launch_bounds__(256) reduce_kernel(const RedDesc *__restrict__ descs) {
    const RedDesc D = descs[blockIdx.x];
    __shared__ double red[8];
    const int nq = D.grad_out ? 2 * D.p + 1 : 1;
    for (int q = 0; q < nq; q++) {
        const int cnt = q == 0 ? D.cntE : (q <= D.p ? D.cntB : D.cntG);
        const double *src = D.part + (int64_t)q * D.stride;
        double acc = 0.0;
        for (int i = threadIdx.x; i < cnt; i += 256) acc += src[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < 8; w++) tot += red[w];
            if (q == 0)
                *D.E_out = tot;
            else
                D.grad_out[q - 1] = 2.0 * tot;
        }
        __syncthreads();
    }
}

template <int T, int BWD, int COST>
cudaError_t launch_one(const PassDesc *d, const uint32_t *tb, int nd, uint32_t tiles, int *err,
                       cudaStream_t s) {
    constexpr int TILE = 1 << T;
    const size_t smem = (size_t)(BWD ? 2 : 1) * TILE * sizeof(float2) + kPhaseTable * sizeof(float2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(xpass_kernel<T, BWD, COST>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    xpass_kernel<T, BWD, COST><<<tiles, 1 << (T - 5), smem, s>>>(d, tb, nd, err);
    return cudaGetLastError();
}

}  // namespace

bool xpass_supported(int T, int bwd) { return (T == 12 || T == 13) || (T == 14 && !bwd); }
int small_max_n() { return kSmallMaxN; }

cudaError_t launch_xpass(int T, int bwd, int cost_dtype, const PassDesc *d, const uint32_t *tb,
                         int nd, uint32_t tiles, int *err, cudaStream_t s) {
    const int c = cost_dtype;
#define QG_X(TT, BB, CC)                                                          \
    if (T == TT && bwd == BB && c == CC) return launch_one<TT, BB, CC>(d, tb, nd, tiles, err, s);
    QG_X(12, 0, 0) QG_X(12, 0, 1) QG_X(12, 1, 0) QG_X(12, 1, 1)
    QG_X(13, 0, 0) QG_X(13, 0, 1) QG_X(13, 1, 0) QG_X(13, 1, 1)
    QG_X(14, 0, 0) QG_X(14, 0, 1)
#undef QG_X
    return cudaErrorInvalidValue;
}

cudaError_t launch_small(const SmallDesc *d, int nd, int cost_dtype, int want_grad, int max_n,
                         int *err, cudaStream_t s) {
    const size_t smem = (size_t)2 * (1u << max_n) * sizeof(float2) + kPhaseTable * sizeof(float2);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nd, kSmallThreads, smem, s>>>(d, err);
        return cudaGetLastError();
    };
    if (cost_dtype == 0) return want_grad ? go(small_kernel<0, 1>) : go(small_kernel<0, 0>);
    return want_grad ? go(small_kernel<1, 1>) : go(small_kernel<1, 0>);
}

cudaError_t launch_prep(const PrepDesc *d, int nd, int *err, cudaStream_t s) {
    prep_kernel<<<nd, 256, 0, s>>>(d, err);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const RedDesc *d, int nd, cudaStream_t s) {
    reduce_kernel<<<nd, 256, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace qg
