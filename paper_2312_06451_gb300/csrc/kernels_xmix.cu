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
//   * Each thread holds 16 amplitudes of each vector in registers (a tile of
//     2^12 amplitudes, 256 threads).  A tile goes through three
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
#include "bulk.cuh"

#include <math.h>

#include <algorithm>

namespace qg {
namespace {

constexpr float kTwoPiF = 6.2831853071795864769f;

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

// (sin, cos) of 2 pi t for a float64 turn count t, without float64
// transcendentals (slow on this part): t = q/4 + r with the nearest quarter
// turn q/4 removed in float64, |r| <= 1/8 to the float32 sincospi, then the
// quarter turns applied exactly.  Values near zero keep their relative accuracy.
__device__ __forceinline__ void sincos_turns(double t, float *s, float *c) {
    const double q = rint(4.0 * t);
    const float r = (float)(t - 0.25 * q);
    float sr, cr;
    sincospif(2.f * r, &sr, &cr);
    switch ((int)((long long)q & 3)) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
    }
}

constexpr double kInvTwoPi = 0.15915494309189533577;  // 1 / (2 pi)

// Round coefficients from one beta (rotation) and the round's gamma.
__device__ __forceinline__ RoundCoef make_coef(double be, double ga) {
    const double bb = be * kInvTwoPi;
    float sb, cb;
    sincos_turns(bb, &sb, &cb);
    RoundCoef c;
    c.cb = cb;
    c.sb = sb;
    // tan form unless cos b is so small that the running 1/cos factors or
    // the pair-term scale would leave float32 range (then: direct form)
    if (fabsf(cb) >= 2.44140625e-4f) {
        c.bmode = 0;
        c.bt = sb / cb;
    } else {
        c.bmode = 2;
        c.bt = 0.f;
    }
    c.rescale = fabsf(cb) < 0.25f ? 1 : 0;
    const double g = ga * kInvTwoPi;
    c.g_hi = (float)g;
    c.g_lo = (float)(g - (double)c.g_hi);
    c.b_hi = (float)bb;
    c.b_lo = (float)(bb - (double)c.b_hi);
    c.pad = 0.f;
    return c;
}

// ----------------------------------------------------------------------------
// Packed (f32x2) rotations in the twisted basis s_x = (-i)^{|x|} psi_x, where
// e^{-i b X} on a qubit is the real matrix [[c, s], [-s, c]] applied to the
// (re, im) pair of both amplitudes alike.  Register pairs (i, i | 1<<RB).
struct Rot {
    float2 tt, ntt;  // (t, t), (-t, -t), t = tan b   (bmode 0)
    float c, s;      // cos b, sin b                  (bmode 2)
    float psc;       // pair-term scale per rotation: c^2 (bmode 0) or 1
    int mode;
};

template <int RB, int MODE>
__device__ __forceinline__ void rot_pairs(float2 (&a)[16], const Rot &R) {
    if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
            if (i & (1 << RB)) continue;
            const int j = i | (1 << RB);
            const float2 x = a[i], y = a[j];
            a[i] = __ffma2_rn(R.tt, y, x);   // s0 + t s1
            a[j] = __ffma2_rn(R.ntt, x, y);  // s1 - t s0
        }
    } else {
        const float2 cc = make_float2(R.c, R.c), ss = make_float2(R.s, R.s), nss = make_float2(-R.s, -R.s);
#pragma unroll
        for (int i = 0; i < 16; i++) {
            if (i & (1 << RB)) continue;
            const int j = i | (1 << RB);
            const float2 x = a[i], y = a[j];
            a[i] = __ffma2_rn(ss, y, __fmul2_rn(cc, x));   // c s0 + s s1
            a[j] = __ffma2_rn(nss, x, __fmul2_rn(cc, y));  // c s1 - s s0
        }
    }
}

// This thread's share of Im <lambda| X_q |psi> in the twisted basis, where
// X_q becomes [[0, i], [-i, 0]]: sum over pairs of l0.p1 - l1.p0 (real dot
// products of (re, im) pairs), with four independent packed accumulators.
template <int RB>
__device__ __forceinline__ float pair_dot(const float2 (&l)[16], const float2 (&p)[16]) {
    float2 ap[4], am[4];
#pragma unroll
    for (int k = 0; k < 4; k++) ap[k] = am[k] = make_float2(0.f, 0.f);
    int k = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        if (i & (1 << RB)) continue;
        const int j = i | (1 << RB);
        ap[k & 3] = __ffma2_rn(l[i], p[j], ap[k & 3]);
        am[k & 3] = __ffma2_rn(l[j], p[i], am[k & 3]);
        k++;
    }
    const float2 sp = __fadd2_rn(__fadd2_rn(ap[0], ap[1]), __fadd2_rn(ap[2], ap[3]));
    const float2 sm = __fadd2_rn(__fadd2_rn(am[0], am[1]), __fadd2_rn(am[2], am[3]));
    return (sp.x + sp.y) - (sm.x + sm.y);
}

// The rotations of one register layout ("stage"): on bit k = register bit k
// carries an active qubit.  The adjoint first takes the pair terms
// <lambda|X_q|psi> of all the stage's qubits at the stage's starting point --
// any point of the round where both vectors have had the same rotations
// gives the same value, because all X_q commute -- and then rotates lambda,
// and psi only when rot_psi is set (its later values are not always needed).
template <int BWD, int MODE>
__device__ __forceinline__ void stage_rot(float2 (&a)[16], float2 (&l)[16], uint32_t on, const Rot &R,
                                          float &pscale, float &bacc, bool rot_psi, bool pairs = true) {
    if (BWD) {
        if (pairs) {
            float s = 0.f;
            if (on & 1u) s += pair_dot<0>(l, a);
            if (on & 2u) s += pair_dot<1>(l, a);
            if (on & 4u) s += pair_dot<2>(l, a);
            if (on & 8u) s += pair_dot<3>(l, a);
            bacc = fmaf(s, pscale, bacc);
        }
        for (uint32_t m = on; m; m &= m - 1u) pscale *= R.psc;
        if (on & 1u) rot_pairs<0, MODE>(l, R);
        if (on & 2u) rot_pairs<1, MODE>(l, R);
        if (on & 4u) rot_pairs<2, MODE>(l, R);
        if (on & 8u) rot_pairs<3, MODE>(l, R);
    }
    if (!BWD || rot_psi) {
        if (on & 1u) rot_pairs<0, MODE>(a, R);
        if (on & 2u) rot_pairs<1, MODE>(a, R);
        if (on & 4u) rot_pairs<2, MODE>(a, R);
        if (on & 8u) rot_pairs<3, MODE>(a, R);
    }
}

// Multi-angle rotations (one angle per qubit): register bit j of the stage
// carries local bit Lj, with rot[Lj] = (cos b, +-sin b, +-tan b, cos^2 b).
// MODE 0 is the tan form (the cosines are applied per stage or per pass like
// the single-angle path, pscale tracks them for the pair terms), MODE 2 the
// direct form.  The adjoint's pair terms go to one accumulator per local bit.
template <int BWD, int MODE, int L0, int L1, int L2, int L3, int NQ>
__device__ __forceinline__ void stage_rot_ma(float2 (&a)[16], float2 (&l)[16], uint32_t on, const float4 *rot,
                                             float (&bq)[NQ], float &pscale, bool rot_psi) {
    Rot R[4];
    const int Ls[4] = {L0, L1, L2, L3};
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float4 q = rot[Ls[j]];
        R[j].c = q.x;
        R[j].s = q.y;
        R[j].tt = make_float2(q.z, q.z);
        R[j].ntt = make_float2(-q.z, -q.z);
    }
    if (BWD) {
        if (on & 1u) bq[L0] = fmaf(pair_dot<0>(l, a), pscale, bq[L0]);
        if (on & 2u) bq[L1] = fmaf(pair_dot<1>(l, a), pscale, bq[L1]);
        if (on & 4u) bq[L2] = fmaf(pair_dot<2>(l, a), pscale, bq[L2]);
        if (on & 8u) bq[L3] = fmaf(pair_dot<3>(l, a), pscale, bq[L3]);
        if (MODE == 0) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (on & (1u << j)) pscale *= rot[Ls[j]].w;
        }
        if (on & 1u) rot_pairs<0, MODE>(l, R[0]);
        if (on & 2u) rot_pairs<1, MODE>(l, R[1]);
        if (on & 4u) rot_pairs<2, MODE>(l, R[2]);
        if (on & 8u) rot_pairs<3, MODE>(l, R[3]);
    }
    if (!BWD || rot_psi) {
        if (on & 1u) rot_pairs<0, MODE>(a, R[0]);
        if (on & 2u) rot_pairs<1, MODE>(a, R[1]);
        if (on & 4u) rot_pairs<2, MODE>(a, R[2]);
        if (on & 8u) rot_pairs<3, MODE>(a, R[3]);
    }
}

// Register bits of the stage whose local bits are b0..b3, from the pass's
// active-qubit mask.
__device__ __forceinline__ uint32_t stage_mask(uint32_t active, int b0, int b1, int b2, int b3) {
    return ((active >> b0) & 1u) | (((active >> b1) & 1u) << 1) | (((active >> b2) & 1u) << 2) |
           (((active >> b3) & 1u) << 3);
}

template <int BWD>
__device__ __forceinline__ void scale_all(float2 (&a)[16], float2 (&l)[16], float f) {
    const float2 ff = make_float2(f, f);
#pragma unroll
    for (int i = 0; i < 16; i++) {
        a[i] = __fmul2_rn(ff, a[i]);
        if (BWD) l[i] = __fmul2_rn(ff, l[i]);
    }
}

// (-i)^k * v
__device__ __forceinline__ float2 twist(float2 v, int k) {
    switch (k & 3) {
    case 0: return v;
    case 1: return make_float2(v.y, -v.x);
    case 2: return make_float2(-v.x, -v.y);
    default: return make_float2(-v.y, v.x);
    }
}

// Float64 arithmetic runs at a small fraction of the float32 rate on this
// part, so the per-tile partial sums below are summed across a warp in
// float32 (a fixed shuffle tree, so still bitwise reproducible) and only the
// warp totals are widened to float64 for the sums over tiles and warps.
// Each thread's share is itself a float32 sum of a few hundred terms, so the
// warp step adds an error of the same order (~1e-7 of the sum of magnitudes).

// Warp sum of one float per lane; every lane gets the total.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of two floats per lane in one tree: the total of x lands in
// lanes 0..15, the total of y in lanes 16..31.
__device__ __forceinline__ float warp_sum2_f(float x, float y) {
    const bool hi = (threadIdx.x & 16u) != 0;
    float v = (hi ? y : x) + __shfl_xor_sync(0xffffffffu, hi ? x : y, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of 16 floats per lane as a reduce-scatter: each step halves the
// values a lane keeps and trades the other half with its partner, so value
// j's total lands in lanes 2j and 2j + 1 after 16 shuffles (not 80).
__device__ __forceinline__ float warp_sum16_f(const float (&v)[16]) {
    const uint32_t lane = threadIdx.x & 31u;
    float w8[8], w4[4], w2[2];
    const bool h4 = lane & 16u, h3 = lane & 8u, h2 = lane & 4u, h1 = lane & 2u;
#pragma unroll
    for (int k = 0; k < 8; k++)
        w8[k] = (h4 ? v[k + 8] : v[k]) + __shfl_xor_sync(0xffffffffu, h4 ? v[k] : v[k + 8], 16);
#pragma unroll
    for (int k = 0; k < 4; k++)
        w4[k] = (h3 ? w8[k + 4] : w8[k]) + __shfl_xor_sync(0xffffffffu, h3 ? w8[k] : w8[k + 4], 8);
#pragma unroll
    for (int k = 0; k < 2; k++)
        w2[k] = (h2 ? w4[k + 2] : w4[k]) + __shfl_xor_sync(0xffffffffu, h2 ? w4[k] : w4[k + 2], 4);
    float w = (h1 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, h1 ? w2[0] : w2[1], 2);
    return w + __shfl_xor_sync(0xffffffffu, w, 1);
}

// Deterministic block sum of one float per thread: float32 within each
// warp, float64 across warps; the result is valid in thread 0.
template <int NW>
__device__ __forceinline__ double block_sum(float v, double *red) {
    double d = (double)warp_sum_f(v);
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

// ----------------------------------------------------------- TMA / mbarrier
// (mbarrier and bulk-copy wrappers: bulk.cuh)
// One TMA tensor copy of a 4-d box (coordinates c0..c3) global -> shared.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// --------------------------------------------------------------------------
// The pass kernel (persistent).  A tile is 2^12 amplitudes; 256 threads hold
// 16 amplitudes each (per vector).  Tile-local bit j is global bit gpos[j]
// (bits 0..c-1 are the contiguous run).  Register layouts (local bits):
//   stage 1: amp bit 0 -> 0 (16-byte pair), lanes -> 1..5, warps -> 6..8,
//            amp bits 1..3 -> 9..11                (read from the TMA buffer)
//   stage 2: amp bits 0..3 -> 1..4, lanes -> {0,6,7,8,5}, warps -> 9..11
//   stage 3: amp bits 0..3 -> 5..8, lanes -> 0..4, warps -> 9..11  (stores)
// Rotated on stage 1: local 0, 9, 10, 11; stage 2: 1..4; stage 3: 5..8.
//
// Pipeline: warp 0 loads the tiles of this CTA with TMA copies into NBUF
// shared-memory buffers (completion on one mbarrier per buffer; the tile's
// descriptor index and base offset travel with it through the barrier); a
// tile is transposed in place in its buffer, which goes back to the loader as
// soon as its last stage has been read.
constexpr int kT = kPassTileBits;
constexpr int kTile = 1 << kT;
constexpr int kNT = 256;
constexpr int kNW = kNT / 32;

template <int BWD, int COST>
struct PassGeom {
    static constexpr uint32_t kPsiB = kTile * 8;
    static constexpr uint32_t kCostB = kTile * (COST == 0 ? 4 : 1);
    static constexpr uint32_t kBufB = kPsiB * (BWD ? 2 : 1) + kCostB;
    static constexpr uint32_t kStashB = (BWD && COST == 0) ? kTile * 4 : 0;  // after the buffers
    // single-buffered adjoint with float costs: buffer 0's cost slot and the
    // stash make one vector's worth of transpose space (see tile_body)
    static constexpr bool kEarly = BWD && COST == 0 && kCostB + kStashB == kPsiB;
    static constexpr uint32_t kHead = 256 + kPhaseTable * 8;  // barriers, tile info, phase table
};

struct TileInfo {
    int di;
    uint32_t tl;    // tile index within the descriptor
    uint32_t base;  // global element offset of local index 0
    uint32_t pad;
};

template <int BWD>
__device__ __forceinline__ bool needs_cost(uint32_t flags) {
    return BWD ? (flags & (PF_LAM_FROM_C | PF_PHASE | PF_FUSED)) != 0 : (flags & (PF_PHASE | PF_E | PF_FUSED)) != 0;
}

// Descriptor of tile t for the loader.  A CTA claims its tiles in
// increasing order, so the search walks forward from the previous answer
// (`cursor`, warp 0's own) for a few descriptors, and bisects when the claim
// jumped further (small descriptors: a CTA's claims are about a grid apart).
__device__ __forceinline__ int next_desc(const uint32_t *__restrict__ tile_begin, int ndesc, uint32_t t,
                                         int &cursor) {
    int di = cursor;
    if (di < 0 || di >= ndesc || t < tile_begin[di]) {
        di = find_desc(tile_begin, ndesc, t);
    } else {
        int steps = 0;
        while (di < ndesc && t >= tile_begin[di + 1] && steps < 4) {
            di++;
            steps++;
        }
        if (di < ndesc && t >= tile_begin[di + 1]) di = find_desc(tile_begin, ndesc, t);
    }
    if (di >= ndesc) di = -1;
    if (di >= 0) cursor = di;
    return di;
}

// Global offset of local index 0 of tile tl: the tile index's bits fill the
// free qubits in increasing order, which are c..lo-1 and lo+h..n-1 for a pass
// keeping qubits 0..c-1 contiguous and gathering lo..lo+h-1 (h = T - c).
__device__ __forceinline__ uint32_t tile_base(uint32_t tl, int c, int lo) {
    if (c >= kT) return tl << kT;
    const int h = kT - c, nb = lo - c;
    const uint32_t hi = lo + h < 32 ? (tl >> nb) << (lo + h) : 0u;  // nothing above a top block
    return ((tl & ((1u << nb) - 1u)) << c) | hi;
}

// Warp 0: start the loads of tile t into buffer buf (all 32 lanes call).
template <int BWD, int COST>
// The descriptor the CTA is working on sits in shared memory (Ds) with its
// tile range and index in s_tr = {first tile, end tile, index}; a next tile in
// that range (the common case) needs no global load at all.
__device__ __forceinline__ void issue_tile(uint32_t t, unsigned char *buf, uint32_t bar, TileInfo *info,
                                           const PassDesc *__restrict__ descs,
                                           const uint32_t *__restrict__ tile_begin, int ndesc, int &cursor,
                                           const PassDesc *Ds, const uint32_t *s_tr) {
    using G = PassGeom<BWD, COST>;
    const int lane = threadIdx.x & 31;
    const bool here = Ds && t >= s_tr[0] && t < s_tr[1];
    const int di = here ? (int)s_tr[2] : next_desc(tile_begin, ndesc, t, cursor);
    fence_proxy_async();
    if (di < 0) {
        if (lane == 0) {
            info->di = -1;
            mbar_arrive_tx(bar, 0);
        }
        return;
    }
    const PassDesc *Dg = here ? Ds : descs + di;
    const uint32_t flags = Dg->flags;
    const int c = Dg->c;
    const uint32_t tl = t - (here ? s_tr[0] : tile_begin[di]);
    const uint32_t base = tile_base(tl, c, Dg->gpos[c < kT ? c : 0]);
    const bool ld_psi = BWD || !(flags & PF_GEN_INIT);
    const bool ld_lam = BWD && !(flags & PF_LAM_FROM_C);
    const bool ld_cost = needs_cost<BWD>(flags);
    const uint32_t bytes = (ld_psi ? G::kPsiB : 0) + (ld_lam ? G::kPsiB : 0) + (ld_cost ? G::kCostB : 0);
    if (lane == 0) {
        info->di = di;
        info->tl = tl;
        info->base = base;
        mbar_arrive_tx(bar, bytes);
    }
    __syncwarp();
    const uint32_t sb = smem_u32(buf);
    const float2 *psi = Dg->psi_in;
    const float2 *lam = Dg->lam_in;
    const unsigned char *cost = static_cast<const unsigned char *>(Dg->cost);
    constexpr uint32_t cb = COST == 0 ? 4 : 1;
    // Gathered tile with a tensor map: one TMA op per operand.  Box = 2^c
    // contiguous elements x 2^(T-c) rows at stride 2^lo; tile coordinates
    // are the free bits below lo (dim 1) and above lo + T - c (dim 3).
    const void *tm_psi = Dg->tm_psi, *tm_lam = Dg->tm_lam, *tm_cost = Dg->tm_cost;
    bool seg_psi = ld_psi, seg_lam = ld_lam, seg_cost = ld_cost;
    if (lane == 0 && (tm_psi || tm_lam || tm_cost)) {
        const int lo = Dg->gpos[c];  // gathered pass: lo > c
        const int c1 = (int)(tl & ((1u << (lo - c)) - 1u)), c3 = (int)(tl >> (lo - c));
        if (ld_psi && tm_psi) tma_load_4d(sb, tm_psi, 0, c1, 0, c3, bar);
        if (ld_lam && tm_lam) tma_load_4d(sb + G::kPsiB, tm_lam, 0, c1, 0, c3, bar);
        if (ld_cost && tm_cost) tma_load_4d(sb + G::kPsiB * (BWD ? 2 : 1), tm_cost, 0, c1, 0, c3, bar);
    }
    seg_psi = seg_psi && !tm_psi;
    seg_lam = seg_lam && !tm_lam;
    seg_cost = seg_cost && !tm_cost;
    if (!(seg_psi || seg_lam || seg_cost)) return;
    const int nseg = 1 << (kT - c);
    const uint32_t segn = 1u << c;
    const int glo = c < kT ? Dg->gpos[c] : 0;  // segment s starts at base + s 2^lo
    for (int s = lane; s < nseg; s += 32) {
        const uint32_t off = base + ((uint32_t)s << glo);
        const uint32_t ls = (uint32_t)s << c;
        if (seg_psi) bulk_g2s(sb + ls * 8, psi + off, segn * 8, bar);
        if (seg_lam) bulk_g2s(sb + G::kPsiB + ls * 8, lam + off, segn * 8, bar);
        if (seg_cost)
            bulk_g2s(sb + G::kPsiB * (BWD ? 2 : 1) + ls * cb, cost + (size_t)off * cb, segn * cb, bar);
    }
}

// Tiles are handed out dynamically: the first NBUF per CTA statically
// (blockIdx + k gridDim), the rest from a per-launch counter in the order CTAs
// ask for them, so CTAs that run faster take more tiles and the launch ends
// with every CTA within about one tile of the others.  Partial sums sit in
// per-tile slots, so the results do not depend on which CTA took a tile.
// A claim past the last tile posts an end marker through the buffer's barrier.
constexpr int kTileEnd = -2;

__device__ __forceinline__ void post_end(uint32_t bar, TileInfo *info) {
    if ((threadIdx.x & 31) == 0) {
        info->di = kTileEnd;
        mbar_arrive_tx(bar, 0);
    }
}

// Constants of the descriptor currently being processed.
struct PassConst {
    Rot R;
    float ghi, glo, amp0;
    float c0;                  // adjoint: cost shift (C - c0 as the operator)
    float fs1, fs2, fs3, fse;  // cos b factors per stage / per pass
    uint32_t flags, active, g3, g1;
    uint32_t rs3[4], rs1[3];
    int rescale;
};

// One tile: stages 1..3, in-place transposes in buffer b, fused epilogue.
// MODE is the rotation form (0 tan, 2 direct); the two forms are separate
// copies of this body so the common one stays compact in the instruction
// cache.  Optional work (initial state, phase, epilogue) sits in loops of its
// own that are skipped as a whole when a pass does not need them.  PAT fixes
// the stages' active-qubit masks at compile time as in the round-boundary
// body (1: all twelve tile bits, 2: tile bits 4..11, 0: from the descriptor);
// the forward passes use it, the adjoint ones would spill.
template <int BWD, int COST, int NBUF, int MODE, int VAR, int PAT>
__device__ __forceinline__ void tile_body(const PassConst &K, const PassDesc &D, const float2 *stab,
                                          const float4 *s_rot, const float4 *s_w,
                                          unsigned char *bufs, int b, uint32_t bar, uint32_t *sched, int cost_free,
                                          uint32_t total, uint32_t base, uint32_t tl, TileInfo *tinfo,
                                          const PassDesc *__restrict__ descs,
                                          const uint32_t *__restrict__ tile_begin, int ndesc, int &cursor,
                                          const uint32_t *s_tr) {
    using G = PassGeom<BWD, COST>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l1 = ((uint32_t)lane << 1) | ((uint32_t)warp << 6);
    const uint32_t l2 = ((uint32_t)lane & 1u) | ((((uint32_t)lane >> 1) & 7u) << 6) |
                        ((((uint32_t)lane >> 4) & 1u) << 5) | ((uint32_t)warp << 9);
    const uint32_t l3 = (uint32_t)lane | ((uint32_t)warp << 9);
    const uint32_t p1 = swz(l1), p2 = swz(l2), p3 = swz(l3);
    const uint32_t flags = K.flags, active = K.active;
    const uint32_t m1 = PAT == 1 ? 0xFu : PAT == 2 ? 0xEu : stage_mask(active, 0, 9, 10, 11),
                   m2 = PAT == 1 ? 0xFu : PAT == 2 ? 0x8u : stage_mask(active, 1, 2, 3, 4),
                   m3 = PAT != 0 ? 0xFu : stage_mask(active, 5, 6, 7, 8);
    // warp 0: claim the next tile for this buffer and start its loads
    auto claim_issue = [&]() {
        uint32_t tn = 0;
        if (lane == 0) tn = (uint32_t)NBUF * gridDim.x + atomicAdd(sched, 1u);
        tn = __shfl_sync(0xffffffffu, tn, 0);
        if (tn < total)
            issue_tile<BWD, COST>(tn, bufs + b * G::kBufB, bar, &tinfo[b], descs, tile_begin, ndesc, cursor, &D,
                                  s_tr);
        else
            post_end(bar, &tinfo[b]);
    };

    float2 *sp = reinterpret_cast<float2 *>(bufs + b * G::kBufB);
    float2 *sl = sp + kTile;
    const unsigned char *scost = bufs + b * G::kBufB + G::kPsiB * (BWD ? 2 : 1);
    float2 a[16];
    float2 l[16];
    float pscale = 1.f, bacc = 0.f;
    constexpr bool MA = VAR == 1;  // multi-angle
    constexpr bool GM = VAR == 2;  // general X mixer: fixed half-round rotations, no pair terms
    float bq[MA ? 12 : 1];         // multi-angle: pair terms per local bit
#pragma unroll
    for (int j = 0; j < (MA ? 12 : 1); j++) bq[j] = 0.f;

    // ---------------- stage 1: read the landed tile
    if (!BWD && (flags & PF_GEN_INIT)) {
        if (GM) {  // the general mixer's passes keep plain amplitudes
#pragma unroll
            for (int i = 0; i < 16; i++) a[i] = make_float2(K.amp0, 0.f);
        } else {
            // uniform state in the twisted basis: amp0 * (-i)^{|x|}, |x| = |base| + |local|
            const float2 a0 = twist(make_float2(K.amp0, 0.f), __popc(base) + __popc(l1));
#pragma unroll
            for (int r = 0; r < 8; r++) {
                a[2 * r] = twist(a0, __popc(r));
                a[2 * r + 1] = twist(a0, __popc(r) + 1);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const float4 v = *reinterpret_cast<const float4 *>(sp + (l1 | ((uint32_t)r << 9)));
            a[2 * r] = make_float2(v.x, v.y);
            a[2 * r + 1] = make_float2(v.z, v.w);
        }
        if (!GM && !BWD && (flags & PF_TWIST_IN)) {
            const float2 w0 = twist(make_float2(1.f, 0.f), __popc(base) + __popc(l1));
#pragma unroll
            for (int r = 0; r < 8; r++) {
                a[2 * r] = cmul(twist(a[2 * r], __popc(r)), w0);
                a[2 * r + 1] = cmul(twist(a[2 * r + 1], __popc(r) + 1), w0);
            }
        }
    }
    if (BWD && !(flags & PF_LAM_FROM_C)) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const float4 v = *reinterpret_cast<const float4 *>(sl + (l1 | ((uint32_t)r << 9)));
            l[2 * r] = make_float2(v.x, v.y);
            l[2 * r + 1] = make_float2(v.z, v.w);
        }
    }
    if (BWD ? (flags & PF_LAM_FROM_C) : (flags & PF_PHASE)) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const uint32_t idx = l1 | ((uint32_t)r << 9);
            float c0, c1;
            if (COST == 0) {
                const float2 cc = *reinterpret_cast<const float2 *>(reinterpret_cast<const float *>(scost) + idx);
                c0 = cc.x;
                c1 = cc.y;
            } else {
                const uchar2 cc = *reinterpret_cast<const uchar2 *>(scost + idx);
                c0 = (float)cc.x;
                c1 = (float)cc.y;
                if (!BWD) {
                    a[2 * r] = cmul(a[2 * r], stab[cc.x]);
                    a[2 * r + 1] = cmul(a[2 * r + 1], stab[cc.y]);
                }
            }
            if (BWD) {
                const float d0 = c0 - K.c0, d1 = c1 - K.c0;
                l[2 * r] = __fmul2_rn(make_float2(d0, d0), a[2 * r]);
                l[2 * r + 1] = __fmul2_rn(make_float2(d1, d1), a[2 * r + 1]);
            } else if (COST == 0) {
                a[2 * r] = cmul(a[2 * r], phase_f32(c0, K.ghi, K.glo));
                a[2 * r + 1] = cmul(a[2 * r + 1], phase_f32(c1, K.ghi, K.glo));
            }
        }
    }
    if (GM && !BWD && (flags & PF_WDIAG)) {
        // general X mixer: e^{-i b G(|x|)} on the global index x of every
        // amplitude (local bits below c stay, the others start at qubit lo)
        const int c = D.c, lo = c < kT ? D.gpos[c] : 0;
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const uint32_t lq = l1 | ((uint32_t)r << 9);
            const uint32_t x = base + (c >= kT ? lq : ((lq & ((1u << c) - 1u)) | ((lq >> c) << lo)));
            const float4 t0 = s_w[__popc(x)], t1 = s_w[__popc(x | 1u)];
            a[2 * r] = cmul(a[2 * r], make_float2(t0.x, t0.y));
            a[2 * r + 1] = cmul(a[2 * r + 1], make_float2(t1.x, t1.y));
        }
    }
    if constexpr (MA) stage_rot_ma<BWD, MODE, 0, 9, 10, 11>(a, l, stage_mask(active, 0, 9, 10, 11), s_rot, bq, pscale, true);
    else stage_rot<BWD, MODE>(a, l, m1, K.R, pscale, bacc, true, !GM);
    if (K.rescale) {
        scale_all<BWD>(a, l, K.fs1);
        pscale = 1.f;
    }

    // ---------------- stage 1 -> 2, in place (swizzled)
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const uint32_t idx = p1 ^ swz((uint32_t)r << 9);
        *reinterpret_cast<float4 *>(sp + idx) = make_float4(a[2 * r].x, a[2 * r].y, a[2 * r + 1].x, a[2 * r + 1].y);
        if (BWD)
            *reinterpret_cast<float4 *>(sl + idx) = make_float4(l[2 * r].x, l[2 * r].y, l[2 * r + 1].x, l[2 * r + 1].y);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        a[i] = sp[p2 ^ ((uint32_t)i << 1)];
        if (BWD) l[i] = sl[p2 ^ ((uint32_t)i << 1)];
    }
    // A single-buffered adjoint tile that reads no cost hands its buffer back
    // here, after the stage-2 read, and runs the warp-private stage 2 -> 3
    // transpose through buffer 0's cost slot and the float-cost stash (32 KB),
    // which no load writes while the launch reads no cost at all (cost_free).
    // The next tile's loads then run under stages 2 and 3 instead of stage 3
    // alone.
    const bool early = G::kEarly && NBUF == 1 && cost_free && !needs_cost<BWD>(flags);
    if (early) {
        __syncthreads();
        if (warp == 0) claim_issue();
    }
    if constexpr (MA) stage_rot_ma<BWD, MODE, 1, 2, 3, 4>(a, l, stage_mask(active, 1, 2, 3, 4), s_rot, bq, pscale, true);
    else stage_rot<BWD, MODE>(a, l, m2, K.R, pscale, bacc, true, !GM);
    if (K.rescale) {
        scale_all<BWD>(a, l, K.fs2);
        pscale = 1.f;
    }

    // ---------------- stage 2 -> 3: local bits 9..11 are the warp index in
    // both layouts and the swizzle moves bits 1..3 only, so each warp reads
    // back just what it wrote: a warp barrier is enough
    if (G::kEarly && NBUF == 1 && early) {
        // one vector at a time through the 32 KB behind buffer 0's vectors
        float2 *scr = reinterpret_cast<float2 *>(bufs + 2 * G::kPsiB);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) scr[p2 ^ ((uint32_t)i << 1)] = a[i];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) a[i] = scr[p3 ^ swz((uint32_t)i << 5)];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) scr[p2 ^ ((uint32_t)i << 1)] = l[i];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) l[i] = scr[p3 ^ swz((uint32_t)i << 5)];
    } else {
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) {
            sp[p2 ^ ((uint32_t)i << 1)] = a[i];
            if (BWD) sl[p2 ^ ((uint32_t)i << 1)] = l[i];
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const uint32_t idx = p3 ^ swz((uint32_t)i << 5);
            a[i] = sp[idx];
            if (BWD) l[i] = sl[idx];
        }
    }
    // Cost values of this thread's stage-3 amplitudes, read before the buffer
    // goes back to the loader: uint8 costs packed four to a register; float
    // costs of the adjoint copied to this thread's own slots of a stash that
    // the loader never writes (16 live registers there cause spills).
    const bool epi_c = BWD ? (flags & PF_PHASE) : (flags & PF_E);
    float cst[16];
    uint32_t cpk[4];
    float *stash = reinterpret_cast<float *>(bufs + NBUF * G::kBufB);
    if (epi_c) {
        if (COST == 1) {
#pragma unroll
            for (int q = 0; q < 4; q++) cpk[q] = 0u;
#pragma unroll
            for (int i = 0; i < 16; i++)
                cpk[i >> 2] |= (uint32_t)scost[l3 | ((uint32_t)i << 5)] << (8 * (i & 3));
        } else if (BWD) {
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const uint32_t ci = l3 | ((uint32_t)i << 5);
                stash[ci] = reinterpret_cast<const float *>(scost)[ci];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; i++)
                cst[i] = reinterpret_cast<const float *>(scost)[l3 | ((uint32_t)i << 5)];
        }
    }
    auto cost_at = [&](int i) -> float {
        if (COST == 1) return (float)((cpk[i >> 2] >> (8 * (i & 3))) & 255u);
        if (BWD) return stash[l3 | ((uint32_t)i << 5)];
        return cst[i];
    };
    // the buffer is consumed: start the tile NBUF ahead
    if (!early) {
        __syncthreads();
        if (warp == 0) claim_issue();
    }
    // psi after the last stage is needed only when it is stored or meets the
    // phase epilogue (the adjoint with per-pass checkpoints stores lambda only)
    const bool psi_live = !BWD || D.psi_out != nullptr || (flags & PF_PHASE) || (GM && (flags & PF_WDIAG));
    if constexpr (MA) stage_rot_ma<BWD, MODE, 5, 6, 7, 8>(a, l, stage_mask(active, 5, 6, 7, 8), s_rot, bq, pscale, psi_live);
    else stage_rot<BWD, MODE>(a, l, m3, K.R, pscale, bacc, psi_live, !GM);
    scale_all<BWD>(a, l, K.rescale ? K.fs3 : K.fse);
    if (GM && BWD && (flags & PF_WDIAG)) {
        // general X mixer: the beta partial sum_x G(|x|) Im(conj(lam) psi) in
        // the frame between the two half rounds, then the diagonal undone
        const uint32_t g0 = base + K.g3;
        float wacc = 0.f;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const uint32_t x = g0 + (((i & 1) ? K.rs3[0] : 0) + ((i & 2) ? K.rs3[1] : 0) + ((i & 4) ? K.rs3[2] : 0) +
                                     ((i & 8) ? K.rs3[3] : 0));
            const float4 t = s_w[__popc(x)];
            wacc = fmaf(t.z, fmaf(l[i].x, a[i].y, -l[i].y * a[i].x), wacc);
            l[i] = cmul_conj(l[i], make_float2(t.x, t.y));
            if (D.psi_out) a[i] = cmul_conj(a[i], make_float2(t.x, t.y));
        }
        bacc += wacc;
    }

    // ---------------- stage 3: fused epilogue, coalesced store
    float eacc = 0.f;
    if (epi_c) {
        if (!BWD) {
#pragma unroll
            for (int i = 0; i < 16; i++) eacc = fmaf(cost_at(i), fmaf(a[i].x, a[i].x, a[i].y * a[i].y), eacc);
        } else {
            const bool un_psi = flags & PF_UNPHASE_PSI;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const float C = cost_at(i);
                const float2 ph = COST == 0 ? phase_f32(C, K.ghi, K.glo) : stab[(int)C];
                eacc = fmaf(C - K.c0, fmaf(l[i].x, a[i].y, -l[i].y * a[i].x), eacc);
                l[i] = cmul_conj(l[i], ph);
                if (un_psi) a[i] = cmul_conj(a[i], ph);
            }
        }
    }
    const uint32_t g = base + K.g3;
    if (D.psi_out) {
        float2 *out = D.psi_out + g;
#pragma unroll
        for (int i = 0; i < 16; i++)
            __stcs(out + (((i & 1) ? K.rs3[0] : 0) + ((i & 2) ? K.rs3[1] : 0) + ((i & 4) ? K.rs3[2] : 0) +
                          ((i & 8) ? K.rs3[3] : 0)),
                   a[i]);
    }
    if (BWD && D.lam_out) {
        float2 *out = D.lam_out + g;
#pragma unroll
        for (int i = 0; i < 16; i++)
            __stcs(out + (((i & 1) ? K.rs3[0] : 0) + ((i & 2) ? K.rs3[1] : 0) + ((i & 4) ? K.rs3[2] : 0) +
                          ((i & 8) ? K.rs3[3] : 0)),
                   l[i]);
    }
    // per-warp partial sums: slot tile * 8 + warp (no block barrier)
    if (BWD) {
        if constexpr (MA) {  // slot (local bit j, tile, warp); j's total in lane 2j
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = j < 12 ? bq[j < 12 ? j : 0] : 0.f;
            const float tb = warp_sum16_f(v);
            const uint32_t j = (uint32_t)lane >> 1;
            if (!(lane & 1) && j < 12u && ((active >> j) & 1u) && D.part_beta)
                D.part_beta[((size_t)j * D.ntiles + tl) * kNW + warp] = (double)tb;
            if (flags & PF_PHASE) {
                const float tg = warp_sum_f(eacc);
                if (lane == 0 && D.part_gamma) D.part_gamma[tl * kNW + warp] = (double)tg;
            }
        } else {  // beta's total in lane 0, gamma's in lane 16
            const float t = warp_sum2_f(bacc, eacc);
            if (lane == 0 && D.part_beta) D.part_beta[tl * kNW + warp] = (double)t;
            if ((flags & PF_PHASE) && lane == 16 && D.part_gamma) D.part_gamma[tl * kNW + warp] = (double)t;
        }
    } else if (flags & PF_E) {
        const float te = warp_sum_f(eacc);
        if (lane == 0 && D.part_E) D.part_E[tl * kNW + warp] = (double)te;
    }
}

// Rotation and phase constants of one round for the tiles of a descriptor
// (K.active must be set): rotation form, the cos factors per stage / per pass.
__device__ __forceinline__ void set_round(PassConst &K, const RoundCoef &cf, float sgn) {
    K.R.mode = cf.bmode;
    K.R.tt = make_float2(sgn * cf.bt, sgn * cf.bt);
    K.R.ntt = make_float2(-sgn * cf.bt, -sgn * cf.bt);
    K.R.c = cf.cb;
    K.R.s = sgn * cf.sb;
    K.R.psc = cf.bmode == 0 ? cf.cb * cf.cb : 1.f;
    K.rescale = (cf.bmode == 0 && cf.rescale) ? 1 : 0;
    const float c = cf.bmode == 0 ? cf.cb : 1.f;
    const int k1 = __popc(K.active & 0xE01u), k2 = __popc(K.active & 0x1Eu), k3 = __popc(K.active & 0x1E0u);
    K.fs1 = K.fs2 = K.fs3 = 1.f;
    for (int k = 0; k < k1; k++) K.fs1 *= c;
    for (int k = 0; k < k2; k++) K.fs2 *= c;
    for (int k = 0; k < k3; k++) K.fs3 *= c;
    K.fse = K.rescale ? 1.f : K.fs1 * K.fs2 * K.fs3;
    K.ghi = cf.g_hi;
    K.glo = cf.g_lo;
}

// Round-boundary tile (PF_FUSED).  The tile's bits are the last qubit group
// of round k and the first of round k+1, so one pass applies round k's
// rotations, the phase of round k+1 and round k+1's rotations (forward), or
// undoes them in reverse order with both rounds' pair terms and the gamma
// partial in between (adjoint).  The register stages run 1 -> 2 -> 3, the
// phase at stage 3 (cost values in the tile buffer, natural order), then back
// 3 -> 2 -> 1 through the inverse transposes, and the result is stored from
// the stage-1 (load) layout as 16-byte pairs.  KA is the round applied first
// (forward: k; adjoint: k+1), KB the second; KP holds the phase (round k+1).
// PAT fixes the stages' active-qubit masks at compile time for the two groups
// the default schedules use most: 1 = all twelve tile bits (the contiguous
// group), 2 = tile bits 4..11 (a gathered group with four contiguous bits);
// 0 takes them from the descriptor.
template <int BWD, int COST, int NBUF, int MA, int MB, int PAT>
__device__ __forceinline__ void tile_body_fused_impl(const PassConst &KA, const PassConst &KB, const PassConst &KP,
                                                uint32_t g1, const uint32_t (&rs1)[3],
                                                const PassDesc &D, const float2 *stab, unsigned char *bufs, int b,
                                                uint32_t bar, uint32_t *sched, uint32_t total, uint32_t base,
                                                uint32_t tl, TileInfo *tinfo, const PassDesc *__restrict__ descs,
                                                const uint32_t *__restrict__ tile_begin, int ndesc, int &cursor,
                                                const uint32_t *s_tr) {
    using G = PassGeom<BWD, COST>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l1 = ((uint32_t)lane << 1) | ((uint32_t)warp << 6);
    const uint32_t l2 = ((uint32_t)lane & 1u) | ((((uint32_t)lane >> 1) & 7u) << 6) |
                        ((((uint32_t)lane >> 4) & 1u) << 5) | ((uint32_t)warp << 9);
    const uint32_t l3 = (uint32_t)lane | ((uint32_t)warp << 9);
    const uint32_t p1 = swz(l1), p2 = swz(l2), p3 = swz(l3);
    const uint32_t active = KA.active;
    float2 *sp = reinterpret_cast<float2 *>(bufs + b * G::kBufB);
    float2 *sl = sp + kTile;
    const unsigned char *scost = bufs + b * G::kBufB + G::kPsiB * (BWD ? 2 : 1);
    float2 a[16], l[16];
    float pscale = 1.f, bA = 0.f, bB = 0.f, eacc = 0.f;
    const uint32_t m1 = PAT == 1 ? 0xFu : PAT == 2 ? 0xEu : stage_mask(active, 0, 9, 10, 11),
                   m2 = PAT == 1 ? 0xFu : PAT == 2 ? 0x8u : stage_mask(active, 1, 2, 3, 4),
                   m3 = PAT != 0 ? 0xFu : stage_mask(active, 5, 6, 7, 8);

    // ---------------- stage 1: read the landed tile
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const float4 v = *reinterpret_cast<const float4 *>(sp + (l1 | ((uint32_t)r << 9)));
        a[2 * r] = make_float2(v.x, v.y);
        a[2 * r + 1] = make_float2(v.z, v.w);
        if (BWD) {
            const float4 w = *reinterpret_cast<const float4 *>(sl + (l1 | ((uint32_t)r << 9)));
            l[2 * r] = make_float2(w.x, w.y);
            l[2 * r + 1] = make_float2(w.z, w.w);
        }
    }
    // ---------------- round A, stages 1 -> 2 -> 3
    stage_rot<BWD, MA>(a, l, m1, KA.R, pscale, bA, true);
    if (KA.rescale) {
        scale_all<BWD>(a, l, KA.fs1);
        pscale = 1.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const uint32_t idx = p1 ^ swz((uint32_t)r << 9);
        *reinterpret_cast<float4 *>(sp + idx) = make_float4(a[2 * r].x, a[2 * r].y, a[2 * r + 1].x, a[2 * r + 1].y);
        if (BWD)
            *reinterpret_cast<float4 *>(sl + idx) = make_float4(l[2 * r].x, l[2 * r].y, l[2 * r + 1].x, l[2 * r + 1].y);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        a[i] = sp[p2 ^ ((uint32_t)i << 1)];
        if (BWD) l[i] = sl[p2 ^ ((uint32_t)i << 1)];
    }
    stage_rot<BWD, MA>(a, l, m2, KA.R, pscale, bA, true);
    if (KA.rescale) {
        scale_all<BWD>(a, l, KA.fs2);
        pscale = 1.f;
    }
    // stage 2 -> 3 inside each warp's 512 amplitudes
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        sp[p2 ^ ((uint32_t)i << 1)] = a[i];
        if (BWD) sl[p2 ^ ((uint32_t)i << 1)] = l[i];
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t idx = p3 ^ swz((uint32_t)i << 5);
        a[i] = sp[idx];
        if (BWD) l[i] = sl[idx];
    }
    stage_rot<BWD, MA>(a, l, m3, KA.R, pscale, bA, true);
    scale_all<BWD>(a, l, KA.rescale ? KA.fs3 : KA.fse);
    pscale = 1.f;

    // ---------------- the phase of round k+1 between the two rounds
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t ci = l3 | ((uint32_t)i << 5);
        const float C = COST == 0 ? reinterpret_cast<const float *>(scost)[ci] : (float)scost[ci];
        const float2 ph = COST == 0 ? phase_f32(C, KP.ghi, KP.glo) : stab[scost[ci]];
        if (BWD) {
            eacc = fmaf(C - KP.c0, fmaf(l[i].x, a[i].y, -l[i].y * a[i].x), eacc);
            l[i] = cmul_conj(l[i], ph);
            a[i] = cmul_conj(a[i], ph);
        } else {
            a[i] = cmul(a[i], ph);
        }
    }

    // ---------------- round B, stages 3 -> 2 -> 1
    stage_rot<BWD, MB>(a, l, m3, KB.R, pscale, bB, true);
    if (KB.rescale) {
        scale_all<BWD>(a, l, KB.fs3);
        pscale = 1.f;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t idx = p3 ^ swz((uint32_t)i << 5);
        sp[idx] = a[i];
        if (BWD) sl[idx] = l[i];
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        a[i] = sp[p2 ^ ((uint32_t)i << 1)];
        if (BWD) l[i] = sl[p2 ^ ((uint32_t)i << 1)];
    }
    stage_rot<BWD, MB>(a, l, m2, KB.R, pscale, bB, true);
    if (KB.rescale) {
        scale_all<BWD>(a, l, KB.fs2);
        pscale = 1.f;
    }
    // stage 2 -> 1: each warp rewrites its own 512 amplitudes, then all read across warps
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        sp[p2 ^ ((uint32_t)i << 1)] = a[i];
        if (BWD) sl[p2 ^ ((uint32_t)i << 1)] = l[i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const uint32_t idx = p1 ^ swz((uint32_t)r << 9);
        const float4 v = *reinterpret_cast<const float4 *>(sp + idx);
        a[2 * r] = make_float2(v.x, v.y);
        a[2 * r + 1] = make_float2(v.z, v.w);
        if (BWD) {
            const float4 w = *reinterpret_cast<const float4 *>(sl + idx);
            l[2 * r] = make_float2(w.x, w.y);
            l[2 * r + 1] = make_float2(w.z, w.w);
        }
    }
    // the buffer is consumed: start the tile NBUF ahead
    __syncthreads();
    if (warp == 0) {
        uint32_t tn = 0;
        if (lane == 0) tn = (uint32_t)NBUF * gridDim.x + atomicAdd(sched, 1u);
        tn = __shfl_sync(0xffffffffu, tn, 0);
        if (tn < total)
            issue_tile<BWD, COST>(tn, bufs + b * G::kBufB, bar, &tinfo[b], descs, tile_begin, ndesc, cursor, &D,
                                  s_tr);
        else
            post_end(bar, &tinfo[b]);
    }
    // psi is dead after the last adjoint stage
    stage_rot<BWD, MB>(a, l, m1, KB.R, pscale, bB, !BWD);
    scale_all<BWD>(a, l, KB.rescale ? KB.fs1 : KB.fse);

    // ---------------- store from the stage-1 layout: 16-byte amplitude pairs
    {
        float2 *out = BWD ? D.lam_out : D.psi_out;
        if (out) {
            const float2 *v = BWD ? l : a;
            out += base + g1;
#pragma unroll
            for (int r = 0; r < 8; r++) {
                const uint32_t o = ((r & 1) ? rs1[0] : 0u) + ((r & 2) ? rs1[1] : 0u) + ((r & 4) ? rs1[2] : 0u);
                __stcs(reinterpret_cast<float4 *>(out + o),
                       make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y));
            }
        }
    }
    if (BWD) {  // round k+1's beta total in lane 0, round k's in lane 16; gamma by its own tree
        const float t = warp_sum2_f(bA, bB);
        if (lane == 0 && D.part_beta) D.part_beta[tl * kNW + warp] = (double)t;
        if (lane == 16 && D.part_beta2) D.part_beta2[tl * kNW + warp] = (double)t;
        const float tg = warp_sum_f(eacc);
        if (lane == 0 && D.part_gamma) D.part_gamma[tl * kNW + warp] = (double)tg;
    }
}

// The common case (both rounds in the tan form, a mask pattern known at
// compile time) inline; the direct form (|cos b| tiny, rare) and other
// groups out of line, so that their registers do not set the register
// allocation of the common path.
template <int BWD, int COST, int NBUF, int MA, int MB, int PAT>
__device__ __forceinline__ void tile_body_fused(const PassConst &KA, const PassConst &KB, const PassConst &KP,
                                                uint32_t g1, const uint32_t (&rs1)[3],
                                                const PassDesc &D, const float2 *stab, unsigned char *bufs, int b,
                                                uint32_t bar, uint32_t *sched, uint32_t total, uint32_t base,
                                                uint32_t tl, TileInfo *tinfo, const PassDesc *__restrict__ descs,
                                                const uint32_t *__restrict__ tile_begin, int ndesc, int &cursor,
                                                const uint32_t *s_tr) {
    tile_body_fused_impl<BWD, COST, NBUF, MA, MB, PAT>(KA, KB, KP, g1, rs1, D, stab, bufs, b, bar, sched, total,
                                                       base, tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
}
template <int BWD, int COST, int NBUF, int MA, int MB>
__device__ __noinline__ void tile_body_fused_rare(const PassConst &KA, const PassConst &KB, const PassConst &KP,
                                                  uint32_t g1, const uint32_t (&rs1)[3],
                                                  const PassDesc &D, const float2 *stab, unsigned char *bufs, int b,
                                                  uint32_t bar, uint32_t *sched, uint32_t total, uint32_t base,
                                                  uint32_t tl, TileInfo *tinfo, const PassDesc *__restrict__ descs,
                                                  const uint32_t *__restrict__ tile_begin, int ndesc, int &cursor,
                                                  const uint32_t *s_tr) {
    tile_body_fused_impl<BWD, COST, NBUF, MA, MB, 0>(KA, KB, KP, g1, rs1, D, stab, bufs, b, bar, sched, total, base,
                                                     tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
}

template <int BWD, int COST, int NBUF, int VAR, int FUSED>
__global__ void __launch_bounds__(kNT, (BWD && NBUF > 1) ? 1 : 2)
xpass_kernel(const PassDesc *__restrict__ descs, const uint32_t *__restrict__ tile_begin, int ndesc,
             uint32_t total, int *err, uint32_t *__restrict__ sched, int cost_free) {
    using G = PassGeom<BWD, COST>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    TileInfo *tinfo = reinterpret_cast<TileInfo *>(smem_raw + 64);
    float2 *stab = reinterpret_cast<float2 *>(smem_raw + 256);
    unsigned char *bufs = smem_raw + G::kHead;
    __shared__ PassDesc D;
    __shared__ float4 s_rot[12];  // multi-angle: (cos, +-sin, +-tan, cos^2) per local bit
    __shared__ float4 s_w[33];    // general X mixer: weight phases and G(w)
    __shared__ uint32_t s_tr[3];  // D's first tile, end tile and index
    __shared__ PassConst s_kf[2];  // round-boundary launches: rounds k and k+1 (uniform fields)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int b = 0; b < NBUF; b++) mbar_init(smem_u32(&bars[b]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t stride = gridDim.x;
    int cursor = 0;  // loader's descriptor search position (warp 0)
    if (warp == 0) {
        for (int k = 0; k < NBUF; k++) {
            const uint32_t t = blockIdx.x + (uint32_t)k * stride;
            if (t < total)
                issue_tile<BWD, COST>(t, bufs + k * G::kBufB, smem_u32(&bars[k]), &tinfo[k], descs, tile_begin,
                                      ndesc, cursor, nullptr, nullptr);
            else
                post_end(smem_u32(&bars[k]), &tinfo[k]);
        }
    }
    const uint32_t l3 = (uint32_t)lane | ((uint32_t)warp << 9);
    int cur = -1;
    PassConst K;

    for (uint32_t it = 0;; it++) {
        const int b = (int)(it % NBUF);
        const uint32_t bar = smem_u32(&bars[b]);
        const bool ok = mbar_wait(bar, (it / NBUF) & 1u);
        const TileInfo ti = tinfo[b];
        if (ok && ti.di == kTileEnd) break;  // uniform; later claims are end markers too
        const int di = ok ? ti.di : -1;
        if (di != cur) {  // uniform: every thread read the same tile info
            __syncthreads();  // the previous tile's epilogue is done with D / stab
            if (di < 0) {
                if (tid == 0) atomicOr(err, ok ? DERR_BAD_DESC : DERR_TIMEOUT);
                // let every load this CTA started land before the block exits
                // (each of the other buffers holds a claimed tile or an end marker)
                for (int k = 1; k < NBUF; k++)
                    mbar_wait(smem_u32(&bars[(it + k) % NBUF]), ((it + k) / NBUF) & 1u);
                if (!ok) mbar_wait(bar, (it / NBUF) & 1u);
                return;
            }
            const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + di);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&D);
            for (int i = tid; i < (int)(sizeof(PassDesc) / 4); i += kNT) dst[i] = src[i];
            if (tid == 0) {
                s_tr[0] = tile_begin[di];
                s_tr[1] = tile_begin[di + 1];
                s_tr[2] = (uint32_t)di;
            }
            __syncthreads();
            K.flags = D.flags;
            K.active = D.active;
            K.amp0 = D.amp0;
            // undoing a round (adjoint) uses the coefficients of -b
            const float sgn = BWD ? -1.f : 1.f;
            set_round(K, *D.coef, sgn);
            K.c0 = (BWD && D.c0 && (K.flags & (PF_LAM_FROM_C | PF_PHASE | PF_FUSED))) ? (float)*D.c0 : 0.f;
            K.g3 = 0;
            for (int j = 0; j < kT; j++)
                if ((l3 >> j) & 1u) K.g3 += 1u << D.gpos[j];
#pragma unroll
            for (int k = 0; k < 4; k++) K.rs3[k] = 1u << D.gpos[5 + k];
            if (FUSED) {  // stage-1 store offsets (round-boundary passes)
                const uint32_t l1s = ((uint32_t)lane << 1) | ((uint32_t)warp << 6);
                K.g1 = 0;
                for (int j = 1; j < 9; j++)
                    if ((l1s >> j) & 1u) K.g1 += 1u << D.gpos[j];
#pragma unroll
                for (int k = 0; k < 3; k++) K.rs1[k] = 1u << D.gpos[9 + k];
            }
            if (FUSED && tid == 0) {  // both rounds of a boundary pass, for every thread
                PassConst K2 = K;
                set_round(K2, *D.coef2, sgn);
                s_kf[0] = K;
                s_kf[1] = K2;
            }
            if (COST == 1 && (K.flags & (PF_PHASE | PF_FUSED)))
                for (int i = tid; i < kPhaseTable; i += kNT) stab[i] = D.table[i];
            if (VAR == 2 && (K.flags & PF_WDIAG))
                for (int i = tid; i <= D.n; i += kNT) s_w[i] = D.wtab[i];
            if (VAR == 1) {
                // per-qubit rotations: D.coef is this round's n entries, indexed
                // by global qubit.  The tan form when every rotated qubit allows
                // it, with the cosines per stage (rescale: any |cos| < 1/4) or
                // once per pass, else the direct form.
                bool tan_ok = true, resc = false;
                if (tid < kT) {
                    const RoundCoef q = D.coef[D.gpos[tid]];
                    s_rot[tid] = make_float4(q.cb, sgn * q.sb, sgn * q.bt, q.cb * q.cb);
                    const bool on = (K.active >> tid) & 1u;
                    tan_ok = !on || q.bmode == 0;
                    resc = on && q.rescale;
                }
                tan_ok = __syncthreads_and(tan_ok);
                resc = __syncthreads_or(resc) && tan_ok;
                auto prod = [&](int b0, int b1, int b2, int b3) {
                    float f = 1.f;
                    const int bs[4] = {b0, b1, b2, b3};
                    for (int j = 0; j < 4; j++)
                        if ((K.active >> bs[j]) & 1u) f *= s_rot[bs[j]].x;
                    return tan_ok ? f : 1.f;
                };
                K.R.mode = tan_ok ? 0 : 2;
                K.rescale = resc ? 1 : 0;
                K.fs1 = prod(0, 9, 10, 11);
                K.fs2 = prod(1, 2, 3, 4);
                K.fs3 = prod(5, 6, 7, 8);
                K.fse = K.rescale ? 1.f : K.fs1 * K.fs2 * K.fs3;
            }
            __syncthreads();
            cur = di;
        }
        if constexpr (FUSED) {
            // forward: round k then round k+1; adjoint: k+1 first; the phase is round k+1's
            const PassConst &KA = s_kf[BWD ? 1 : 0], &KB = s_kf[BWD ? 0 : 1], &KP = s_kf[1];
            const int mk = (KA.R.mode == 0 ? 0 : 1) | (KB.R.mode == 0 ? 0 : 2);
            if (mk == 0 && KA.active == 0xFFFu)
                tile_body_fused<BWD, COST, NBUF, 0, 0, 1>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                          total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                          cursor, s_tr);
            else if (mk == 0 && KA.active == 0xFF0u)
                tile_body_fused<BWD, COST, NBUF, 0, 0, 2>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                          total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                          cursor, s_tr);
            else if (mk == 0)
                tile_body_fused_rare<BWD, COST, NBUF, 0, 0>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                            total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                            cursor, s_tr);
            else if (mk == 1)
                tile_body_fused_rare<BWD, COST, NBUF, 2, 0>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                            total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                            cursor, s_tr);
            else if (mk == 2)
                tile_body_fused_rare<BWD, COST, NBUF, 0, 2>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                            total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                            cursor, s_tr);
            else
                tile_body_fused_rare<BWD, COST, NBUF, 2, 2>(KA, KB, KP, K.g1, K.rs1, D, stab, bufs, b, bar, sched,
                                                            total, ti.base, ti.tl, tinfo, descs, tile_begin, ndesc,
                                                            cursor, s_tr);
        } else if constexpr (VAR == 0 && !BWD) {  // (adjoint copies spill: measured slower)
            if (K.R.mode == 0 && K.active == 0xFFFu)
                tile_body<BWD, COST, NBUF, 0, 0, 1>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                    ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
            else if (K.R.mode == 0 && K.active == 0xFF0u)
                tile_body<BWD, COST, NBUF, 0, 0, 2>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                    ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
            else if (K.R.mode == 0)
                tile_body<BWD, COST, NBUF, 0, 0, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                    ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
            else
                tile_body<BWD, COST, NBUF, 2, 0, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                    ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
        } else if (VAR == 1 && K.R.mode == 0)
            tile_body<BWD, COST, NBUF, 0, 1, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total, ti.base,
                                                ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
        else if (VAR == 1)
            tile_body<BWD, COST, NBUF, 2, 1, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total, ti.base,
                                                ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
        else if (K.R.mode == 0)
            tile_body<BWD, COST, NBUF, 0, VAR, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                  ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
        else
            tile_body<BWD, COST, NBUF, 2, VAR, 0>(K, D, stab, s_rot, s_w, bufs, b, bar, sched, cost_free, total,
                                                  ti.base, ti.tl, tinfo, descs, tile_begin, ndesc, cursor, s_tr);
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
    extern __shared__ __align__(128) unsigned char smem_raw[];
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

    // general X mixer (plain basis here): H^n diag(e^{-i b d_|x|}) H^n
    __shared__ float2 s_gph[kSmallMaxN + 1];
    auto hadamard_all = [&](float2 *v) {
        const float r = 0.70710678118654752f;
        for (int q = 0; q < n; q++) {
            __syncthreads();
            for (int j = tid; j < H; j += kSmallThreads) {
                const int lo = j & ((1 << q) - 1);
                const int x0 = ((j - lo) << 1) | lo, x1 = x0 | (1 << q);
                const float2 u = v[x0], w = v[x1];
                v[x0] = make_float2(r * (u.x + w.x), r * (u.y + w.y));
                v[x1] = make_float2(r * (u.x - w.x), r * (u.y - w.y));
            }
        }
        __syncthreads();
    };
    auto weight_phases = [&](double b) {  // s_gph[w] = e^{-i b d_w}
        __syncthreads();
        if (tid <= n) {
            float sn, cs;
            sincos_turns(b * D.wts[tid] * kInvTwoPi, &sn, &cs);
            s_gph[tid] = make_float2(cs, -sn);
        }
        __syncthreads();
    };
    // coefficients of round k: one entry, one per qubit (multi-angle) or two
    // (general X mixer); nb angles per round's mixer
    const int nb = D.nq ? D.nq : 1;
    const int cs = D.nq ? D.nq : (D.wts ? 2 : 1);
    auto qcoef = [&](int k, int q) -> const RoundCoef & { return D.coef[k * cs + (D.nq ? q : 0)]; };

    for (int x = tid; x < N; x += kSmallThreads)
        psi[x] = D.init ? D.init[x] : make_float2(D.amp0, 0.f);
    for (int k = 0; k < p; k++) {
        const RoundCoef cf = D.coef[k * cs];
        __syncthreads();
        load_table(k);
        for (int x = tid; x < N; x += kSmallThreads) psi[x] = cmul(psi[x], phase(x, cf));
        if (D.wts) {
            weight_phases(D.angles_beta[k]);
            hadamard_all(psi);
            for (int x = tid; x < N; x += kSmallThreads) psi[x] = cmul(psi[x], s_gph[__popc(x)]);
            hadamard_all(psi);
            continue;
        }
        for (int q = 0; q < n; q++) {
            __syncthreads();
            mix(psi, q, qcoef(k, q).cb, qcoef(k, q).sb);
        }
    }
    __syncthreads();
    float e = 0.f;
    for (int x = tid; x < N; x += kSmallThreads)
        e = fmaf(costv(x), fmaf(psi[x].x, psi[x].x, psi[x].y * psi[x].y), e);
    const double E = block_sum<kSmallThreads / 32>(e, s_red);
    if (tid == 0) *D.E_out = E;
    if constexpr (GRAD) {
    // the adjoint uses C - <C>: the same gradient, without the common
    // component <C> psi in lambda
    __shared__ float s_c0;
    if (tid == 0) s_c0 = (float)E;
    __syncthreads();
    const float c0 = s_c0;
    for (int x = tid; x < N; x += kSmallThreads) {
        const float c = costv(x) - c0;
        lam[x] = make_float2(c * psi[x].x, c * psi[x].y);
    }
    for (int k = p - 1; k >= 0; k--) {
        const RoundCoef cf = D.coef[k * cs];
        __syncthreads();
        float gb = 0.f;
        if (D.wts) {
            // in the Hadamard frame: beta partial sum_z d_|z| Im(conj(lam) psi),
            // then the diagonal undone and the frame left again
            weight_phases(D.angles_beta[k]);
            hadamard_all(lam);
            hadamard_all(psi);
            for (int x = tid; x < N; x += kSmallThreads) {
                const float2 l = lam[x], a = psi[x];
                gb = fmaf((float)D.wts[__popc(x)], l.x * a.y - l.y * a.x, gb);
                lam[x] = cmul_conj(l, s_gph[__popc(x)]);
                psi[x] = cmul_conj(a, s_gph[__popc(x)]);
            }
            const double GB = block_sum<kSmallThreads / 32>(gb, s_red);
            if (tid == 0) D.grad_out[k] = 2.0 * GB;
            hadamard_all(lam);
            hadamard_all(psi);
        }
        for (int q = 0; q < (D.wts ? 0 : n); q++) {
            float gq = 0.f;
            for (int j = tid; j < H; j += kSmallThreads) {
                const int lo = j & ((1 << q) - 1);
                const int x0 = ((j - lo) << 1) | lo, x1 = x0 | (1 << q);
                const float2 l0 = lam[x0], l1 = lam[x1], a0 = psi[x0], a1 = psi[x1];
                gq += l0.x * a1.y - l0.y * a1.x + l1.x * a0.y - l1.y * a0.x;
            }
            if (D.nq) {  // one partial per qubit
                const double GQ = block_sum<kSmallThreads / 32>(gq, s_red);
                if (tid == 0) D.grad_out[k * n + q] = 2.0 * GQ;
            } else {
                gb += gq;
            }
        }
        if (!D.nq && !D.wts) {
            const double GB = block_sum<kSmallThreads / 32>(gb, s_red);
            if (tid == 0) D.grad_out[k] = 2.0 * GB;
        }
        for (int q = 0; q < (D.wts ? 0 : n); q++) {
            __syncthreads();
            mix(lam, q, qcoef(k, q).cb, -qcoef(k, q).sb);
            mix(psi, q, qcoef(k, q).cb, -qcoef(k, q).sb);
        }
        __syncthreads();
        load_table(k);
        float gg = 0.f;
        for (int x = tid; x < N; x += kSmallThreads) {
            const float2 l = lam[x], a = psi[x];
            gg = fmaf(costv(x) - c0, l.x * a.y - l.y * a.x, gg);
        }
        const double GG = block_sum<kSmallThreads / 32>(gg, s_red);
        if (tid == 0) D.grad_out[p * nb + k] = 2.0 * GG;
        for (int x = tid; x < N; x += kSmallThreads) {
            const float2 ph = phase(x, cf);
            lam[x] = cmul_conj(lam[x], ph);
            psi[x] = cmul_conj(psi[x], ph);
        }
    }
    }  // GRAD
}

// --------------------------------------------------------------------------
// n = 12: the whole state is one tile of the pass kernels (256 threads x 16
// amplitudes), so one CTA per angle set runs every round with the pass
// kernels' three register stages and two swizzled transposes; between rounds
// the state waits in shared memory in natural order, never in global memory.
// Same twisted basis as the pass kernels (every qubit is a tile bit, so the
// stage masks are full).  The adjoint undoes each round on psi as well.
struct Round12 {
    Rot R;
    int rescale;
    float fs, fse;  // cos factors: per stage (4 rotations), per round (12)
    float ghi, glo;
};

__device__ __forceinline__ Round12 round12(const RoundCoef &cf, float sgn) {
    Round12 r;
    r.R.mode = cf.bmode;
    r.R.tt = make_float2(sgn * cf.bt, sgn * cf.bt);
    r.R.ntt = make_float2(-sgn * cf.bt, -sgn * cf.bt);
    r.R.c = cf.cb;
    r.R.s = sgn * cf.sb;
    r.R.psc = cf.bmode == 0 ? cf.cb * cf.cb : 1.f;
    r.rescale = (cf.bmode == 0 && cf.rescale) ? 1 : 0;
    const float c = cf.bmode == 0 ? cf.cb : 1.f;
    r.fs = c * c * c * c;
    r.fse = r.rescale ? 1.f : r.fs * r.fs * r.fs;
    r.ghi = cf.g_hi;
    r.glo = cf.g_lo;
    return r;
}

// One round on the state in shared memory (natural order in and out).
// Forward: phase on load (initial state generated or twisted in when first),
// rotations; last: <C> partial, and (GRAD) lambda = C psi written to sl.
// Adjoint: rotations of lambda and psi undone with the pair terms, then the
// gamma partial and the phase undone on both.
template <int BWD, int COST, int MODE>
__device__ void tile12_round(float2 *sp, float2 *sl, const float2 *stab, const void *scost, const SmallDesc &D,
                             const Round12 &rc, bool first, bool last, float c0, float &bacc, float &eacc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t l1 = ((uint32_t)lane << 1) | ((uint32_t)warp << 6);
    const uint32_t l2 = ((uint32_t)lane & 1u) | ((((uint32_t)lane >> 1) & 7u) << 6) |
                        ((((uint32_t)lane >> 4) & 1u) << 5) | ((uint32_t)warp << 9);
    const uint32_t l3 = (uint32_t)lane | ((uint32_t)warp << 9);
    const uint32_t p1 = swz(l1), p2 = swz(l2), p3 = swz(l3);
    auto costv = [&](uint32_t x) -> float {  // the cost vector, copied to shared memory
        if (COST == 0) return reinterpret_cast<const float *>(scost)[x];
        return (float)reinterpret_cast<const unsigned char *>(scost)[x];
    };
    auto phase = [&](uint32_t x) -> float2 {
        if (COST == 0) return phase_f32(costv(x), rc.ghi, rc.glo);
        return stab[reinterpret_cast<const unsigned char *>(scost)[x]];
    };
    float2 a[16], l[16];
    float pscale = 1.f;
    // ---- stage 1: local bits {0, 9, 10, 11} in registers
    if (!BWD && first && !D.init) {
        const float2 a0 = twist(make_float2(D.amp0, 0.f), __popc(l1));
#pragma unroll
        for (int r = 0; r < 8; r++) {
            a[2 * r] = twist(a0, __popc(r));
            a[2 * r + 1] = twist(a0, __popc(r) + 1);
        }
    } else {
        const float2 *src = (!BWD && first) ? D.init : sp;
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const float4 v = *reinterpret_cast<const float4 *>(src + (l1 | ((uint32_t)r << 9)));
            a[2 * r] = make_float2(v.x, v.y);
            a[2 * r + 1] = make_float2(v.z, v.w);
        }
        if (!BWD && first) {
            const float2 w0 = twist(make_float2(1.f, 0.f), __popc(l1));
#pragma unroll
            for (int r = 0; r < 8; r++) {
                a[2 * r] = cmul(twist(a[2 * r], __popc(r)), w0);
                a[2 * r + 1] = cmul(twist(a[2 * r + 1], __popc(r) + 1), w0);
            }
        }
    }
    if (BWD) {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const float4 v = *reinterpret_cast<const float4 *>(sl + (l1 | ((uint32_t)r << 9)));
            l[2 * r] = make_float2(v.x, v.y);
            l[2 * r + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const uint32_t x = l1 | ((uint32_t)r << 9);
            a[2 * r] = cmul(a[2 * r], phase(x));
            a[2 * r + 1] = cmul(a[2 * r + 1], phase(x | 1u));
        }
    }
    stage_rot<BWD, MODE>(a, l, 0xFu, rc.R, pscale, bacc, true);
    if (rc.rescale) {
        scale_all<BWD>(a, l, rc.fs);
        pscale = 1.f;
    }
    // ---- stage 1 -> 2 (in place, swizzled; crosses warps)
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const uint32_t idx = p1 ^ swz((uint32_t)r << 9);
        *reinterpret_cast<float4 *>(sp + idx) = make_float4(a[2 * r].x, a[2 * r].y, a[2 * r + 1].x, a[2 * r + 1].y);
        if (BWD)
            *reinterpret_cast<float4 *>(sl + idx) = make_float4(l[2 * r].x, l[2 * r].y, l[2 * r + 1].x, l[2 * r + 1].y);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        a[i] = sp[p2 ^ ((uint32_t)i << 1)];
        if (BWD) l[i] = sl[p2 ^ ((uint32_t)i << 1)];
    }
    stage_rot<BWD, MODE>(a, l, 0xFu, rc.R, pscale, bacc, true);
    if (rc.rescale) {
        scale_all<BWD>(a, l, rc.fs);
        pscale = 1.f;
    }
    // ---- stage 2 -> 3 (inside each warp's 512-amplitude block)
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        sp[p2 ^ ((uint32_t)i << 1)] = a[i];
        if (BWD) sl[p2 ^ ((uint32_t)i << 1)] = l[i];
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t idx = p3 ^ swz((uint32_t)i << 5);
        a[i] = sp[idx];
        if (BWD) l[i] = sl[idx];
    }
    stage_rot<BWD, MODE>(a, l, 0xFu, rc.R, pscale, bacc, true);
    scale_all<BWD>(a, l, rc.rescale ? rc.fs : rc.fse);
    // ---- epilogue and natural-order store (still this warp's block)
    if (BWD) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const uint32_t x = l3 | ((uint32_t)i << 5);
            const float C = costv(x);
            const float2 ph = phase(x);
            eacc = fmaf(C - c0, fmaf(l[i].x, a[i].y, -l[i].y * a[i].x), eacc);
            l[i] = cmul_conj(l[i], ph);
            a[i] = cmul_conj(a[i], ph);
        }
    } else if (last) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const float C = costv(l3 | ((uint32_t)i << 5));
            eacc = fmaf(C, fmaf(a[i].x, a[i].x, a[i].y * a[i].y), eacc);
        }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 16; i++) {
        sp[l3 | ((uint32_t)i << 5)] = a[i];
        if (BWD) sl[l3 | ((uint32_t)i << 5)] = l[i];
    }
    __syncthreads();
}

template <int COST, int GRAD>
__global__ void __launch_bounds__(kNT) tile12_kernel(const SmallDesc *__restrict__ descs, int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *sp = reinterpret_cast<float2 *>(smem_raw);
    float2 *sl = sp + kTile;
    float2 *stab = sl + kTile;
    unsigned char *scost = reinterpret_cast<unsigned char *>(stab + kPhaseTable);
    __shared__ double s_red[2][kNW];
    const SmallDesc D = descs[blockIdx.x];
    const int p = D.p, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {  // cost vector to shared memory (16-byte words)
        const int words = kTile * (COST == 0 ? 4 : 1) / 16;
        for (int i = tid; i < words; i += kNT)
            reinterpret_cast<uint4 *>(scost)[i] = __ldg(reinterpret_cast<const uint4 *>(D.cost) + i);
        __syncthreads();
    }
    // coefficients and the uint8 phase table come from the angles here (no
    // separate preparation launch); every thread forms the round's coefficients
    const double *ang = D.angles_beta;
    if (tid < 2 * p && !isfinite(ang[tid])) atomicOr(err, DERR_BAD_ANGLE);
    auto load_table = [&](int k) {  // the previous round ended with a block barrier
        if (COST == 1) {
            for (int i = tid; i < kPhaseTable; i += kNT) {
                float sn, cs;
                sincos_turns(ang[p + k] * kInvTwoPi * (double)i, &sn, &cs);
                stab[i] = make_float2(cs, -sn);
            }
            __syncthreads();
        }
    };
    // fixed-order block sums of two per-thread values: float32 within a
    // warp (x in lanes 0..15, y in 16..31), float64 across warps
    auto block_sum2 = [&](float x, float y, double &X, double &Y) {
        const float t = warp_sum2_f(x, y);
        if (lane == 0) s_red[0][warp] = (double)t;
        if (lane == 16) s_red[1][warp] = (double)t;
        __syncthreads();
        X = 0.0;
        Y = 0.0;
        for (int w = 0; w < kNW; w++) {
            X += s_red[0][w];
            Y += s_red[1][w];
        }
        __syncthreads();
    };
    float bacc = 0.f, eacc = 0.f;
    for (int k = 0; k < p; k++) {
        const Round12 rc = round12(make_coef(ang[k], ang[p + k]), 1.f);
        load_table(k);
        if (rc.R.mode == 0)
            tile12_round<0, COST, 0>(sp, sl, stab, scost, D, rc, k == 0, k == p - 1, 0.f, bacc, eacc);
        else
            tile12_round<0, COST, 2>(sp, sl, stab, scost, D, rc, k == 0, k == p - 1, 0.f, bacc, eacc);
    }
    double E, unused;
    block_sum2(eacc, 0.f, E, unused);
    if (tid == 0) *D.E_out = E;
    if constexpr (GRAD) {
        // lambda_p = (C - <C>) psi_p: the adjoint with the cost shifted by its
        // expectation gives the same gradient without the common component
        // <C> psi in lambda (every thread holds E after block_sum2)
        const float c0 = (float)E;
        for (int x = tid; x < kTile; x += kNT) {
            const float C = COST == 0 ? reinterpret_cast<const float *>(scost)[x]
                                      : (float)reinterpret_cast<const unsigned char *>(scost)[x];
            const float2 v = sp[x];
            sl[x] = make_float2((C - c0) * v.x, (C - c0) * v.y);
        }
        __syncthreads();
        for (int k = p - 1; k >= 0; k--) {
            const Round12 rc = round12(make_coef(ang[k], ang[p + k]), -1.f);
            load_table(k);
            float b = 0.f, g = 0.f;
            if (rc.R.mode == 0)
                tile12_round<1, COST, 0>(sp, sl, stab, scost, D, rc, false, false, c0, b, g);
            else
                tile12_round<1, COST, 2>(sp, sl, stab, scost, D, rc, false, false, c0, b, g);
            double B, Gm;
            block_sum2(b, g, B, Gm);
            if (tid == 0) {
                D.grad_out[k] = 2.0 * B;
                D.grad_out[p + k] = 2.0 * Gm;
            }
        }
    }
}

// --------------------------------------------------------------------------
// Angles -> per-round coefficients and uint8 phase tables (float64 math).

__global__ void __launch_bounds__(256) prep_kernel(const PrepDesc *__restrict__ descs, int *err) {
    const PrepDesc D = descs[blockIdx.x];
    // nb angles per round's mixer (nq qubits for multi-angle, else 1):
    // beta_{k,q} = angles[k nb + q], gamma_k = angles[p nb + k]
    const int nb = D.nq ? D.nq : 1;
    for (int e = threadIdx.x; e < (D.gm_n ? 0 : D.p * nb); e += blockDim.x) {
        const int k = e / nb;
        const double be = D.angles[e], ga = D.angles[D.p * nb + k];
        if (!isfinite(be) || !isfinite(ga)) atomicOr(err, DERR_BAD_ANGLE);
        const RoundCoef c = make_coef(be, ga);
        D.coef[e] = c;
    }
    if (D.gm_n) {
        // general X mixer: its passes keep plain (untwisted) amplitudes, on
        // which the real rotation [[c, s], [-s, c]] is e^{i t Y}; e^{i (pi/4) Y}
        // on every qubit takes X_S to Z_S, so e^{-i b f(X)} is the rotation by
        // t = pi/4 (coefficient 2k, with gamma_k), e^{-i b d_|x|}, and the
        // rotation by t = -pi/4 (coefficient 2k + 1)
        const int n = D.gm_n;
        for (int e = threadIdx.x; e < 2 * D.p; e += blockDim.x) {
            const int k = e >> 1;
            const double ga = D.angles[D.p + k];
            if (!isfinite(D.angles[k]) || !isfinite(ga)) atomicOr(err, DERR_BAD_ANGLE);
            RoundCoef c;
            sincos_turns((e & 1) ? -0.125 : 0.125, &c.sb, &c.cb);  // t = -+pi/4
            c.bmode = 2;
            c.bt = 0.f;
            c.rescale = 0;
            const double g = ga * kInvTwoPi;
            c.g_hi = (float)g;
            c.g_lo = (float)(g - (double)c.g_hi);
            c.b_hi = c.b_lo = c.pad = 0.f;
            D.coef[e] = c;
        }
        for (int e = threadIdx.x; e < D.p * (n + 1); e += blockDim.x) {
            const int k = e / (n + 1), w = e - k * (n + 1);
            const double G = D.wts[w];
            float sn, cs;
            sincos_turns(D.angles[k] * G * kInvTwoPi, &sn, &cs);
            D.wtab[e] = make_float4(cs, -sn, (float)G, 0.f);
        }
    }
    if (D.table) {
        const int tot = D.p * D.tsize;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int k = e / D.tsize, cst = e - k * D.tsize;
            // e^{-i gamma c} from the turn count gamma c / (2 pi)
            float s, c;
            sincos_turns(D.angles[D.p * nb + k] * kInvTwoPi * (double)cst, &s, &c);
            D.table[k * kPhaseTable + cst] = make_float2(c, -s);
        }
    }
}

// Fixed-order two-level reduction of the per-(tile, warp) partial sums.
__global__ void __launch_bounds__(256) reduce1_kernel(const RedChunk *__restrict__ chunks, double *level2) {
    __shared__ double red[8];
    const RedChunk C = chunks[blockIdx.x];
    double acc = 0.0;
    for (int i = threadIdx.x; i < C.cnt; i += 256) acc += C.src[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; w++) tot += red[w];
        level2[blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(32) reduce2_kernel(const RedOut *__restrict__ outs, const double *level2) {
    const RedOut O = outs[blockIdx.x];
    double acc = 0.0;
    for (int i = threadIdx.x; i < O.n; i += 32) acc += level2[O.first + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *O.out = O.scale * acc;
}

template <int BWD, int COST, int NBUF, int VAR, int FUSED>
cudaError_t launch_one(const PassDesc *d, const uint32_t *tb, int nd, uint32_t tiles, int *err, uint32_t *sched,
                       int cost_free, cudaStream_t s) {
    using G = PassGeom<BWD, COST>;
    const size_t smem = G::kHead + (size_t)NBUF * G::kBufB + G::kStashB;
    // per device: the shared-memory attribute and the persistent grid size
    static int attr_done[kMaxDevices];
    static int grid_caps[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    e = smem_attr_once(xpass_kernel<BWD, COST, NBUF, VAR, FUSED>, (int)smem, attr_done);
    if (e != cudaSuccess) return e;
    int grid_cap = __atomic_load_n(&grid_caps[dev], __ATOMIC_ACQUIRE);
    if (!grid_cap) {
        int nsm = 0, per_sm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xpass_kernel<BWD, COST, NBUF, VAR, FUSED>, kNT, smem);
        if (e != cudaSuccess) return e;
        grid_cap = std::max(1, nsm * std::max(1, per_sm));
        __atomic_store_n(&grid_caps[dev], grid_cap, __ATOMIC_RELEASE);
    }
    const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)grid_cap);
    xpass_kernel<BWD, COST, NBUF, VAR, FUSED><<<grid, kNT, smem, s>>>(d, tb, nd, tiles, err, sched, cost_free);
    return cudaGetLastError();
}

// One thread waits, with the pass kernels' bounded wait, for a barrier phase
// that no thread and no copy ever completes: the wait gives up, the error word
// records it, and the kernel returns.
__global__ void wait_probe_kernel(int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
    if (!mbar_wait(smem_u32(&bar), 0u)) atomicOr(err, DERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_probe(int *err, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(err);
    return cudaGetLastError();
}

int small_max_n() { return kSmallMaxN; }

template <int VAR, int FUSED>
cudaError_t launch_xpass_t(int bwd, int cost_dtype, int nbuf, const PassDesc *d, const uint32_t *tb, int nd,
                           uint32_t tiles, int *err, uint32_t *sched, int cf, cudaStream_t s) {
    if (!bwd) return cost_dtype == 0 ? launch_one<0, 0, 2, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s)
                                     : launch_one<0, 1, 2, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s);
    // adjoint: one tile buffer and two CTAs per SM (128 registers a thread),
    // or two buffers and one CTA per SM (no register cap below 255)
    if (nbuf == 2)
        return cost_dtype == 0 ? launch_one<1, 0, 2, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s)
                               : launch_one<1, 1, 2, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s);
    return cost_dtype == 0 ? launch_one<1, 0, 1, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s)
                           : launch_one<1, 1, 1, VAR, FUSED>(d, tb, nd, tiles, err, sched, cf, s);
}

cudaError_t launch_xpass(int bwd, int cost_dtype, int nbuf, int var, const PassDesc *d, const uint32_t *tb,
                         int nd, uint32_t tiles, int *err, uint32_t *sched, int cost_free, int fused, cudaStream_t s) {
    if (tiles == 0) return cudaSuccess;
    if (!sched) return cudaErrorInvalidValue;
    if (fused) {  // round-boundary passes: transverse field only
        if (var != 0) return cudaErrorInvalidValue;
        return launch_xpass_t<0, 1>(bwd, cost_dtype, nbuf, d, tb, nd, tiles, err, sched, cost_free, s);
    }
    if (var == 1) return launch_xpass_t<1, 0>(bwd, cost_dtype, nbuf, d, tb, nd, tiles, err, sched, cost_free, s);
    if (var == 2) return launch_xpass_t<2, 0>(bwd, cost_dtype, nbuf, d, tb, nd, tiles, err, sched, cost_free, s);
    return launch_xpass_t<0, 0>(bwd, cost_dtype, nbuf, d, tb, nd, tiles, err, sched, cost_free, s);
}

cudaError_t launch_small(const SmallDesc *d, int nd, int cost_dtype, int want_grad, int max_n,
                         int *err, cudaStream_t s) {
    const size_t smem = (size_t)2 * (1u << max_n) * sizeof(float2) + kPhaseTable * sizeof(float2);
    // the opt-in shared-memory size is raised once per kernel to the largest
    // size any call needs (n <= kSmallMaxN)
    const size_t smem_max = (size_t)2 * (1u << kSmallMaxN) * sizeof(float2) + kPhaseTable * sizeof(float2);
    auto go = [&](auto kern, int slot) -> cudaError_t {
        static int attr_done[4][kMaxDevices];
        cudaError_t e = smem_attr_once(kern, (int)smem_max, attr_done[slot]);
        if (e != cudaSuccess) return e;
        kern<<<nd, kSmallThreads, smem, s>>>(d, err);
        return cudaGetLastError();
    };
    if (cost_dtype == 0) return want_grad ? go(small_kernel<0, 1>, 0) : go(small_kernel<0, 0>, 1);
    return want_grad ? go(small_kernel<1, 1>, 2) : go(small_kernel<1, 0>, 3);
}

cudaError_t launch_tile12(const SmallDesc *d, int nd, int cost_dtype, int want_grad, int *err, cudaStream_t s) {
    const size_t smem = (size_t)2 * kTile * sizeof(float2) + kPhaseTable * sizeof(float2) +
                        (size_t)kTile * (cost_dtype == 0 ? 4 : 1);
    auto go = [&](auto kern, int slot) -> cudaError_t {
        static int attr_done[4][kMaxDevices];
        cudaError_t e = smem_attr_once(kern, (int)smem, attr_done[slot]);
        if (e != cudaSuccess) return e;
        kern<<<nd, kNT, smem, s>>>(d, err);
        return cudaGetLastError();
    };
    if (cost_dtype == 0) return want_grad ? go(tile12_kernel<0, 1>, 0) : go(tile12_kernel<0, 0>, 1);
    return want_grad ? go(tile12_kernel<1, 1>, 2) : go(tile12_kernel<1, 0>, 3);
}

cudaError_t launch_prep(const PrepDesc *d, int nd, int *err, cudaStream_t s) {
    prep_kernel<<<nd, 256, 0, s>>>(d, err);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const RedChunk *chunks, int nchunks, double *level2, const RedOut *outs, int nouts,
                          cudaStream_t s) {
    reduce1_kernel<<<nchunks, 256, 0, s>>>(chunks, level2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce2_kernel<<<nouts, 32, 0, s>>>(outs, level2);
    return cudaGetLastError();
}

}  // namespace qg
