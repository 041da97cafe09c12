// Constrained mixers through a stored eigendecomposition (arXiv 2312.06451,
// Sec. 2.1 and 2.2): H_M = V diag(lambda) V^T on the D feasible states, so
// e^{-i b H_M} = V e^{-i b lambda} V^T and the time goes into the products with
// V and V^T (Sec. 2.2).  V is real orthogonal (H_M real symmetric).
//
// Layout: all angle sets of a group are the columns of the GEMM right-hand
// side.  A state matrix is set-major with real and imaginary parts split:
// row 2s holds Re psi_s, row 2s+1 holds Im psi_s, each of length ld (D padded
// to a multiple of 128 with zeros), so every GEMM operand is K-contiguous.
// V and V^T are kept as padded row-major copies (K-major A operands).
//
// One round (forward):  Y = e^{-i b lambda} (V^T X)       (GEMM 1 + epilogue)
//                       X = e^{-i g' C} (V Y)             (GEMM 2 + epilogue)
// with g' the next round's gamma (the phase separator of round k+1 rides on
// round k's second product).  The adjoint round needs one product per
// direction as well, thanks to checkpoints of V^T phi_k and psi_{k-1}.
#include "common.cuh"

#include <type_traits>

#include <cuda.h>
#include <math.h>

namespace qg {
namespace {

constexpr float kTwoPiF = 6.2831853071795864769f;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// e^{-i 2 pi (g_hi + g_lo) (x_hi + x_lo)} with the product formed as a float
// pair and its integer part removed exactly (|g x| < 2^22).
__device__ __forceinline__ float2 turn_phase(float ghi, float glo, float xhi, float xlo) {
    const float th = ghi * xhi;
    const float te = fmaf(ghi, xhi, -th);
    const float tl = fmaf(ghi, xlo, fmaf(glo, xhi, te));
    const float f = (th - rintf(th)) + tl;
    float s, c;
    __sincosf(kTwoPiF * f, &s, &c);
    return make_float2(c, -s);
}

// --------------------------------------------------------------- SIMT GEMM
// out^T[N][M] = A[M][K] * B^T[N][K]^T, fp32, CUDA cores.  Block tile 128 x 128
// x 16, 256 threads, each a 8 x 8 register tile split into 4 x 4 quadrants
// (rows ty*4.., 64+ty*4..; cols tx*4.., 64+tx*4..), so every 4 consecutive
// columns hold two complete (Re, Im) pairs for the epilogue.
constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

struct EpiArgs {
    int kind;             // EigEpi
    int M;                // valid rows (D)
    int ld;               // row length of state matrices (padded D)
    int nsets;            // valid sets (columns / 2)
    float *out;           // [2S][ld]
    float *out2;          // second output (L = C psi on the last forward round)
    float *ckpt;          // checkpoint written before the phase (or nullptr)
    const float *ck_in;   // checkpoint read by the adjoint epilogues
    const float *lam_hi, *lam_lo;  // eigenvalues split in two floats (padded)
    const void *cost;     // D cost values
    int cost_dtype;
    const RoundCoef *coef;  // per set: coef[s * coef_stride + round]
    int coef_stride;
    int round;            // round whose beta / gamma this epilogue uses
    double *part;         // partial sums [set][M tile] (kind dependent) or nullptr
    int part_stride;      // = number of M tiles
    float *out_lo;        // split outputs for tensor-core operands: out holds the
    float *out2_lo;       // tf32 head, out_lo the float32 remainder (or nullptr)
    const double *c0;     // cost shift of the adjoint (C - c0), or nullptr
};

// Store v to out (and its tf32 split when out_lo is set).  The head is v
// rounded to the nearest tf32 value (magnitude rounded half up on the 13
// dropped bits), so the remainder's sign does not follow v's: the tensor
// cores' own truncation of the remainder then carries no bias.
__device__ __forceinline__ void put(float *out, float *out_lo, size_t o, float v) {
    if (out_lo) {
        const float hi = __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
        out[o] = hi;
        out_lo[o] = v - hi;
    } else {
        out[o] = v;
    }
}

__device__ __forceinline__ float cost_at(const EpiArgs &E, int j) {
    return E.cost_dtype == 0 ? __ldg(reinterpret_cast<const float *>(E.cost) + j)
                             : (float)__ldg(reinterpret_cast<const unsigned char *>(E.cost) + j);
}

// Epilogue on one complex element (row j, set s) given the product value v.
// Returns the contribution to this set's partial sum.
__device__ __forceinline__ float epi_elem(const EpiArgs &E, int j, int s, float2 v) {
    const size_t o_re = (size_t)(2 * s) * E.ld + j, o_im = o_re + E.ld;
    const RoundCoef cf = E.coef[s * E.coef_stride + E.round];
    float contrib = 0.f;
    switch (E.kind) {
    case EPI_STORE:
        put(E.out, E.out_lo, o_re, v.x);
        put(E.out, E.out_lo, o_im, v.y);
        break;
    case EPI_FWD_EIG: {  // Y = e^{-i b lambda} v, checkpoint V^T phi
        if (E.ckpt) {
            E.ckpt[o_re] = v.x;
            E.ckpt[o_im] = v.y;
        }
        const float2 w = cmul(v, turn_phase(cf.b_hi, cf.b_lo, E.lam_hi[j], E.lam_lo[j]));
        put(E.out, E.out_lo, o_re, w.x);
        put(E.out, E.out_lo, o_im, w.y);
        break;
    }
    case EPI_FWD_PHASE: {  // X = e^{-i g' C} v, checkpoint psi_k
        if (E.ckpt) {
            E.ckpt[o_re] = v.x;
            E.ckpt[o_im] = v.y;
        }
        const float2 w = cmul(v, turn_phase(cf.g_hi, cf.g_lo, cost_at(E, j), 0.f));
        put(E.out, E.out_lo, o_re, w.x);
        put(E.out, E.out_lo, o_im, w.y);
        break;
    }
    case EPI_FWD_LAST: {  // psi_p: <C> partial, store psi_p and lambda_p = (C - c0) psi_p
        const float C = cost_at(E, j);
        contrib = C * fmaf(v.x, v.x, v.y * v.y);
        if (E.out) {
            E.out[o_re] = v.x;
            E.out[o_im] = v.y;
        }
        if (E.out2) {
            const float Cs = C - (E.c0 ? (float)__ldg(E.c0) : 0.f);
            put(E.out2, E.out2_lo, o_re, Cs * v.x);
            put(E.out2, E.out2_lo, o_im, Cs * v.y);
        }
        break;
    }
    case EPI_BWD_EIG: {  // beta partial, then undo e^{-i b lambda}
        const float2 ph = turn_phase(cf.b_hi, cf.b_lo, E.lam_hi[j], E.lam_lo[j]);
        const float2 y = make_float2(E.ck_in[o_re], E.ck_in[o_im]);
        const float2 psi = cmul(y, ph);  // V^T psi_k
        const float lam = E.lam_hi[j] + E.lam_lo[j];
        contrib = lam * (v.x * psi.y - v.y * psi.x);  // Im(conj(v) lambda psi)
        const float2 w = make_float2(fmaf(v.x, ph.x, v.y * ph.y), fmaf(v.y, ph.x, -v.x * ph.y));  // v conj(ph)
        put(E.out, E.out_lo, o_re, w.x);
        put(E.out, E.out_lo, o_im, w.y);
        break;
    }
    case EPI_BWD_PHASE: {  // gamma partial with phi = e^{-i g C} psi_{k-1}, then undo the phase
        const float C = cost_at(E, j);
        const float2 ph = turn_phase(cf.g_hi, cf.g_lo, C, 0.f);
        const float2 phi = cmul(make_float2(E.ck_in[o_re], E.ck_in[o_im]), ph);
        contrib = (C - (E.c0 ? (float)__ldg(E.c0) : 0.f)) * (v.x * phi.y - v.y * phi.x);
        if (E.out) {
            const float2 w = make_float2(fmaf(v.x, ph.x, v.y * ph.y), fmaf(v.y, ph.x, -v.x * ph.y));
            put(E.out, E.out_lo, o_re, w.x);
            put(E.out, E.out_lo, o_im, w.y);
        }
        break;
    }
    default:
        break;
    }
    return contrib;
}

__global__ void __launch_bounds__(NT, 2)
gemm_simt_kernel(const float *__restrict__ A, const float *__restrict__ B, int Kp, int lda, int ldb,
                 EpiArgs E, const GroupTile *__restrict__ gt) {
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];
    __shared__ float red[BN / 2][17];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    // tile geometry: a plain product tiles the whole matrix; a grouped
    // (block-diagonal) one takes its block's rows and K range from the table
    int a_row = blockIdx.x * BM, k_off = 0, kext = Kp, m0 = blockIdx.x * BM, row_end = E.M, pidx = blockIdx.x;
    if (gt) {
        const GroupTile g = gt[blockIdx.x];
        a_row = g.a_row;
        k_off = g.k_off;
        kext = g.kext;
        m0 = g.out_row;
        row_end = g.row_end;
        pidx = g.part_idx;
    }
    const int n0 = blockIdx.y * BN;
    // global -> register staging: each thread loads 8 floats of A and of B
    const int lr = tid >> 1, lk = (tid & 1) * 8;
    const float *Ag = A + (size_t)(a_row + lr) * lda + lk;
    const float *Bg = B + (size_t)(n0 + lr) * ldb + k_off + lk;
    float4 ra0, ra1, rb0, rb1;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;

    auto gload = [&](int k0) {
        ra0 = __ldg(reinterpret_cast<const float4 *>(Ag + k0));
        ra1 = __ldg(reinterpret_cast<const float4 *>(Ag + k0 + 4));
        rb0 = __ldg(reinterpret_cast<const float4 *>(Bg + k0));
        rb1 = __ldg(reinterpret_cast<const float4 *>(Bg + k0 + 4));
    };
    auto sstore = [&](int buf) {
        const float va[8] = {ra0.x, ra0.y, ra0.z, ra0.w, ra1.x, ra1.y, ra1.z, ra1.w};
        const float vb[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
#pragma unroll
        for (int q = 0; q < 8; q++) {
            As[buf][lk + q][lr] = va[q];
            Bs[buf][lk + q][lr] = vb[q];
        }
    };
    const int nk = kext / BK;
    gload(0);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nk; kt++) {
        const int cur = kt & 1;
        if (kt + 1 < nk) gload((kt + 1) * BK);
#pragma unroll
        for (int k = 0; k < BK; k++) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) {
            sstore(cur ^ 1);
            __syncthreads();
        }
    }

    // epilogue: rows m = m0 + {ty*4+i, 64+ty*4+i}, cols n = n0 + {tx*4+j, 64+tx*4+j}
    float part[4] = {0.f, 0.f, 0.f, 0.f};  // per owned set (2 per column quad)
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (m >= row_end) continue;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int nc = n0 + (q < 2 ? tx * 4 + 2 * q : 64 + tx * 4 + 2 * (q - 2));
            const int s = nc >> 1;
            if (s >= E.nsets) continue;
            const int jj = q < 2 ? 2 * q : 4 + 2 * (q - 2);
            part[q] += epi_elem(E, m, s, make_float2(acc[i][jj], acc[i][jj + 1]));
        }
    }
    if (E.part) {
        // per-set sums over the 16 thread rows (ty), fixed order
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int sl = q < 2 ? tx * 2 + q : 32 + tx * 2 + (q - 2);  // set within the tile
            red[sl][ty] = part[q];
        }
        __syncthreads();
        if (tid < BN / 2) {
            double t = 0.0;
            for (int r = 0; r < 16; r++) t += (double)red[tid][r];
            const int s = n0 / 2 + tid;
            if (s < E.nsets) E.part[(size_t)s * E.part_stride + pidx] = t;
        }
    }
}

// ------------------------------------------------- tcgen05 split-TF32 GEMM
// out^T[N][M] = A[M][K] B[N][K]^T with A = A_hi + A_lo and B = B_hi + B_lo held
// as separate tf32 planes: per k-step the tensor cores add A_lo B_hi + A_hi B_lo
// + A_hi B_hi ("3xTF32") into a float32 accumulator in tensor memory.
//
// The tensor-core accumulation does not round to nearest: its error shrinks
// magnitudes and grows with the number of products accumulated.  So each
// 32-wide K chunk (12 MMAs) is accumulated into a fresh tensor-memory buffer
// (two buffers alternate) and drained at once into float32 registers with
// round-to-nearest adds.  The operand split rounds the head to nearest (see
// put()), so the hardware's truncation of the tf32 remainders is unbiased.
// Measured on the 12870-state ring mixer at p = 6: <C> within 6.2e-6
// (relative) of the complex128 result; a truncated head gave 1.35e-5.
//
// 128 x 128 output tile per CTA, STAGES-deep TMA ring of 128-byte-swizzled
// K-major tiles.  Warp 0 lane 0 issues TMA loads, warp 1 lane 0 the MMAs;
// warps 2..17 drain the chunks and run the fused epilogue, four per quarter
// of the accumulator rows (a warp reaches only its quarter of tensor memory),
// 32 columns each.  Four accumulator buffers (all 512 tensor-memory columns)
// let the MMAs run up to three chunks ahead of the drain.
// Split of the last, partial wave of tiles along K (see gemm_tc_kernel).
struct SplitArgs {
    int full;       // tiles computed whole, by blocks 0 .. full-1
    int nseg;       // K segments of each remaining tile (1: none)
    float *ws;      // [remaining tile][segment][128 x 128] partial accumulators
    unsigned *cnt;  // [remaining tile] segments finished; zero between products
};

namespace tc {
constexpr int NACC = 4, NDRAIN = 16;  // 128-column accumulators in TMEM, draining warps
// Both products: GNACC buffers, each a pair of TMEM accumulators (the
// A_hi B_hi products, and the two small cross terms apart, so the large sum
// takes only one truncating add per 8-wide K step), drained into the float32
// registers (round to nearest) every DGRP K chunks.  The truncating adds bias
// <C> low in proportion to the adds between drains: on DkS n=16, k=8 (block
// ring mixer, p=6) the error relative to max(|E|, rms C) is about -2.3e-6 -
// 1.45e-6 DGRP; a single accumulator drained every chunk gave -5.9e-6.
constexpr int GNACC = 2, DGRP = 3;
constexpr int BM = 128, BN = 128, BKF = 32, STAGES = 3, NT = 32 * (2 + NDRAIN);
constexpr uint32_t kTileA = BM * 128, kTileB = BN * 128;
constexpr uint32_t kStage = 2 * kTileA + 2 * kTileB;  // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kSmem = STAGES * kStage + 1024;      // + alignment slack
constexpr uint32_t kTmemCols = NACC * BN;               // four 128-column accumulators
static_assert(GNACC * 2 * BN <= (int)kTmemCols, "accumulator pairs exceed the TMEM allocation");
constexpr uint32_t kSpin = 1u << 24;
// instruction descriptor: D f32, A/B tf32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t cnt) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait: gives up after kWaitLimitNs of global time (or kSpin polls).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kSpin; i++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i == 0) t0 = global_ns();
        else if ((i & 15u) == 0u && global_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *m, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(m), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), fixed constant 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // fixed 0b001
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// 32 lanes x 32 bits, 16 consecutive columns per lane (no wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
}  // namespace tc

// The angle pair an epilogue kind turns by: beta for the eigenvalue phases,
// gamma for the cost phases (both in turns, as float32 head and tail).
__device__ __forceinline__ float2 epi_angle(const EpiArgs &E, int s) {
    const RoundCoef &cf = E.coef[s * E.coef_stride + E.round];
    return (E.kind == EPI_FWD_EIG || E.kind == EPI_BWD_EIG) ? make_float2(cf.b_hi, cf.b_lo)
                                                            : make_float2(cf.g_hi, cf.g_lo);
}

// Sums v[q] over the warp's 32 lanes for each of 16 sets with 16 shuffles:
// every exchange halves the values a lane holds (a transposed butterfly).
// Lanes 2i and 2i+1 return the total of set i.
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane) {
    float w[8];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; i++)
        w[i] = (b4 ? v[i + 8] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 8], 16);
#pragma unroll
    for (int i = 0; i < 4; i++)
        w[i] = (b3 ? w[i + 4] : w[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w[i] : w[i + 4], 8);
#pragma unroll
    for (int i = 0; i < 2; i++)
        w[i] = (b2 ? w[i + 2] : w[i]) + __shfl_xor_sync(0xffffffffu, b2 ? w[i] : w[i + 2], 4);
    float t = (b1 ? w[1] : w[0]) + __shfl_xor_sync(0xffffffffu, b1 ? w[0] : w[1], 2);
    return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

// Epilogue of one draining thread in the grouped product: row m, the 16 sets
// s0 .. s0+15 (complex values acc[2q], acc[2q+1]), the same element arithmetic
// as epi_elem.  The row's eigenvalue or cost is loaded once, the angles come
// from shared memory, and the adjoint's checkpoint values are loaded 4 sets at
// a time before those sets' stores, so the thread waits for four round trips to
// memory, not one per set.  c[q] receives set q's partial-sum term.
template <int KIND>
__device__ __forceinline__ void epi_row16(const EpiArgs &E, int m, int s0, int nq, const float2 *ang,
                                          const float *acc, float (&c)[16]) {
    constexpr bool kEig = KIND == EPI_FWD_EIG || KIND == EPI_BWD_EIG;
    constexpr bool kBwd = KIND == EPI_BWD_EIG || KIND == EPI_BWD_PHASE;
    constexpr bool kShift = KIND == EPI_FWD_LAST || KIND == EPI_BWD_PHASE;
    float xh = 0.f, xl = 0.f, c0 = 0.f;
    if (nq <= 0) {  // row past the block, or no valid set
#pragma unroll
        for (int q = 0; q < 16; q++) c[q] = 0.f;
        return;
    }
    if (kEig) {
        xh = __ldg(E.lam_hi + m);
        xl = __ldg(E.lam_lo + m);
    } else if (KIND != EPI_STORE) {
        xh = cost_at(E, m);
    }
    if (kShift && E.c0) c0 = (float)__ldg(E.c0);
    // groups of kGrp sets: the adjoint's checkpoint values of a group are loaded
    // together (groups of 8 spill at this kernel's register cap and measured slower)
    constexpr int kGrp = 4;
#pragma unroll
    for (int h = 0; h < 16; h += kGrp) {
        float2 y[kGrp];
        if (kBwd) {
#pragma unroll
            for (int i = 0; i < kGrp; i++) {
                const size_t o = (size_t)(2 * (s0 + h + i)) * E.ld + m;
                y[i] = h + i < nq ? make_float2(__ldcg(E.ck_in + o), __ldcg(E.ck_in + o + E.ld))
                                  : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int i = 0; i < kGrp; i++) {
            const int q = h + i;
            c[q] = 0.f;
            if (q >= nq) continue;
            const size_t o_re = (size_t)(2 * (s0 + q)) * E.ld + m, o_im = o_re + E.ld;
            const float2 v = make_float2(acc[2 * q], acc[2 * q + 1]);
            if (KIND == EPI_STORE) {
                put(E.out, E.out_lo, o_re, v.x);
                put(E.out, E.out_lo, o_im, v.y);
            } else if (KIND == EPI_FWD_EIG || KIND == EPI_FWD_PHASE) {
                if (E.ckpt) {
                    E.ckpt[o_re] = v.x;
                    E.ckpt[o_im] = v.y;
                }
                const float2 w = cmul(v, turn_phase(ang[q].x, ang[q].y, xh, xl));
                put(E.out, E.out_lo, o_re, w.x);
                put(E.out, E.out_lo, o_im, w.y);
            } else if (KIND == EPI_FWD_LAST) {
                c[q] = xh * fmaf(v.x, v.x, v.y * v.y);
                if (E.out) {
                    E.out[o_re] = v.x;
                    E.out[o_im] = v.y;
                }
                if (E.out2) {
                    const float Cs = xh - c0;
                    put(E.out2, E.out2_lo, o_re, Cs * v.x);
                    put(E.out2, E.out2_lo, o_im, Cs * v.y);
                }
            } else {  // adjoint: partial with the checkpoint turned forward, then undo the phase on v
                const float2 ph = turn_phase(ang[q].x, ang[q].y, xh, xl);
                const float2 f = cmul(y[i], ph);
                c[q] = (kEig ? xh + xl : xh - c0) * (v.x * f.y - v.y * f.x);
                if (kEig || E.out) {
                    const float2 w = make_float2(fmaf(v.x, ph.x, v.y * ph.y), fmaf(v.y, ph.x, -v.x * ph.y));
                    put(E.out, E.out_lo, o_re, w.x);
                    put(E.out, E.out_lo, o_im, w.y);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(tc::NT, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
               const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int Kp, int ntn,
               EpiArgs E, SplitArgs SP, int *err, const GroupTile *__restrict__ gt) {
    using tc::BKF;
    using tc::kStage;
    using tc::kTileA;
    using tc::kTileB;
    using tc::STAGES;
    constexpr int TBM = tc::BM, TBN = tc::BN;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf[tc::GNACC], acce[tc::GNACC];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float red[4][TBN / 2];
    __shared__ float2 s_ang[TBN / 2];  // per-set angles of the tile
    __shared__ int s_last;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // blocks below SP.full take a whole tile; the rest take one K segment of
    // one of the remaining tiles
    int tile = blockIdx.x, seg = 0, nsegs = 1;
    if ((int)blockIdx.x >= SP.full) {
        const int u = blockIdx.x - SP.full;
        tile = SP.full + u / SP.nseg;
        seg = u % SP.nseg;
        nsegs = SP.nseg;
    }
    const int mt = tile / ntn, nt = tile % ntn;
    const int n0 = nt * TBN;
    // plain product: the whole matrix in 128 x 128 tiles; grouped product
    // (block-diagonal A): the block's rows, K range and valid rows from the table
    int m0 = mt * TBM, a_row = mt * TBM, k_off = 0, kext = Kp, row_end = E.M, pidx = mt;
    if (gt) {
        const GroupTile g = gt[mt];
        m0 = g.out_row;
        a_row = g.a_row;
        k_off = g.k_off;
        kext = g.kext;
        row_end = g.row_end;
        pidx = g.part_idx;
    }
    const int nk_all = kext / BKF;
    if (tid >= 64 && tid - 64 < TBN / 2 && n0 / 2 + tid - 64 < E.nsets && E.kind != EPI_STORE &&
        E.kind != EPI_FWD_LAST)
        s_ang[tid - 64] = epi_angle(E, n0 / 2 + tid - 64);  // read after the block barriers below
    const int kb0 = (int)((int64_t)nk_all * seg / nsegs);
    const int nk = (int)((int64_t)nk_all * (seg + 1) / nsegs) - kb0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_base)),
                     "r"(tc::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < STAGES; s++) {
            tc::mbar_init(tc::su32(&full[s]), 1);
            tc::mbar_init(tc::su32(&empty[s]), 1);
        }
        for (int b = 0; b < tc::GNACC; b++) {
            tc::mbar_init(tc::su32(&accf[b]), 1);
            tc::mbar_init(tc::su32(&acce[b]), tc::NDRAIN);  // one arrive per draining warp
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    int issued = 0;  // stages the producer has started (for a clean exit on timeout)
    constexpr int kCols = TBN / (tc::NDRAIN / 4);  // accumulator columns per draining warp
    float acc[kCols];               // its part of one accumulator row

    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; kb++) {
                const int s = kb % STAGES;
                if (kb >= STAGES && !tc::mbar_wait(tc::su32(&empty[s]), ((kb / STAGES) & 1) ^ 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                const uint32_t base = tc::su32(smem + s * kStage);
                const uint32_t fb = tc::su32(&full[s]);
                tc::mbar_expect(fb, kStage);
                const int kx = (kb0 + kb) * BKF;
                tc::tma_2d(base, &tmAh, kx, a_row, fb);
                tc::tma_2d(base + kTileA, &tmAl, kx, a_row, fb);
                tc::tma_2d(base + 2 * kTileA, &tmBh, k_off + kx, n0, fb);
                tc::tma_2d(base + 2 * kTileA + kTileB, &tmBl, k_off + kx, n0, fb);
                issued = kb + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; kb++) {
                const int s = kb % STAGES, a = kb / tc::DGRP, b = a % tc::GNACC;
                const bool first = kb % tc::DGRP == 0, last = kb % tc::DGRP == tc::DGRP - 1 || kb == nk - 1;
                if (first && a >= tc::GNACC && !tc::mbar_wait(tc::su32(&acce[b]), ((a / tc::GNACC) & 1) ^ 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                if (!tc::mbar_wait(tc::su32(&full[s]), (kb / STAGES) & 1)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                tc::fence_after();
                const uint32_t base = tc::su32(smem + s * kStage);
                const uint32_t d = tmem + (uint32_t)(b * 2 * TBN), dc = d + (uint32_t)TBN;
#pragma unroll
                for (int kk = 0; kk < BKF / 8; kk++) {
                    const uint64_t ah = tc::sdesc(base + kk * 32), al = tc::sdesc(base + kTileA + kk * 32);
                    const uint64_t bh = tc::sdesc(base + 2 * kTileA + kk * 32),
                                   bl = tc::sdesc(base + 2 * kTileA + kTileB + kk * 32);
                    const uint32_t accum = (first && kk == 0) ? 0u : 1u;
                    tc::mma_tf32(dc, al, bh, tc::kIdesc, accum);
                    tc::mma_tf32(dc, ah, bl, tc::kIdesc, 1u);
                    tc::mma_tf32(d, ah, bh, tc::kIdesc, accum);
                }
                tc::mma_commit(tc::su32(&empty[s]));
                if (last) tc::mma_commit(tc::su32(&accf[b]));
            }
        }
    } else {
        // draining warps: warp w reads accumulator rows (TMEM lanes) 32 (w % 4) ..
        // and columns kCols * ch .. (ch = which of the quarter's warps)
        const uint32_t lrow = (uint32_t)((warp & 3) * 32) << 16;
        const int ch = (warp - 2) >> 2;
#pragma unroll
        for (int c = 0; c < kCols; c++) acc[c] = 0.f;
        for (int a = 0; a < (nk + tc::DGRP - 1) / tc::DGRP; a++) {
            const int b = a % tc::GNACC;
            if (!tc::mbar_wait(tc::su32(&accf[b]), (a / tc::GNACC) & 1)) {
                atomicExch(&s_fail, 1);
                break;
            }
            tc::fence_after();
#pragma unroll
            for (int q = 0; q < kCols / 16; q++) {  // 16 columns of the pair at a time
                uint32_t r[16], rc[16];
                const uint32_t col = tmem + lrow + (uint32_t)(b * 2 * TBN + ch * kCols + 16 * q);
                tc::tmem_ld16(col, r);
                tc::tmem_ld16(col + TBN, rc);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; i++) acc[16 * q + i] += __uint_as_float(r[i]) + __uint_as_float(rc[i]);
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(tc::su32(&acce[b]));
        }
    }
    __syncwarp();
    const bool failed = __syncthreads_or(s_fail) != 0;
    bool do_epi = !failed;
    if (failed) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        // let started loads land before the block exits
        if (warp == 0 && lane == 0)
            for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; kb++)
                tc::mbar_wait(tc::su32(&full[kb % STAGES]), (kb / STAGES) & 1);
    } else if (nsegs > 1) {
        // K segment of a split tile: store the partial accumulator; the
        // segment that finishes last adds all partials in segment order (the
        // same sum whichever finishes last) and runs the epilogue.  No block
        // ever waits for another.
        const int ti = tile - SP.full;
        float *slots = SP.ws + (size_t)ti * nsegs * (TBM * TBN);
        const int r = (warp & 3) * 32 + lane, c0 = ((warp - 2) >> 2) * kCols;
        if (warp >= 2) {
            float *dst = slots + (size_t)seg * (TBM * TBN) + (size_t)r * TBN + c0;
#pragma unroll
            for (int c = 0; c < kCols; c++) dst[c] = acc[c];
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&SP.cnt[ti], 1u);
            s_last = prev == (unsigned)(nsegs - 1) ? 1 : 0;
            if (s_last) atomicExch(&SP.cnt[ti], 0u);  // ready for the next product
        }
        __syncthreads();
        do_epi = s_last != 0;
        if (do_epi && warp >= 2) {
            __threadfence();
#pragma unroll
            for (int c = 0; c < kCols; c++) {
                float v = 0.f;
                for (int g = 0; g < nsegs; g++) v += __ldcg(slots + (size_t)g * (TBM * TBN) + (size_t)r * TBN + c0 + c);
                acc[c] = v;
            }
        }
    }
    if (do_epi && warp >= 2) {
        static_assert(kCols == 32, "the epilogue takes 16 sets per thread");
        const int rq = warp & 3, ch = (warp - 2) >> 2;
        const int m = m0 + rq * 32 + lane;
        const int s0 = n0 / 2 + ch * (kCols / 2);  // first of this thread's sets
        const int nq = m < row_end ? min(kCols / 2, E.nsets - s0) : 0;
        const float2 *ang = &s_ang[ch * (kCols / 2)];
        float c[kCols / 2];
        switch (E.kind) {
        case EPI_STORE: epi_row16<EPI_STORE>(E, m, s0, nq, ang, acc, c); break;
        case EPI_FWD_EIG: epi_row16<EPI_FWD_EIG>(E, m, s0, nq, ang, acc, c); break;
        case EPI_FWD_PHASE: epi_row16<EPI_FWD_PHASE>(E, m, s0, nq, ang, acc, c); break;
        case EPI_FWD_LAST: epi_row16<EPI_FWD_LAST>(E, m, s0, nq, ang, acc, c); break;
        case EPI_BWD_EIG: epi_row16<EPI_BWD_EIG>(E, m, s0, nq, ang, acc, c); break;
        default: epi_row16<EPI_BWD_PHASE>(E, m, s0, nq, ang, acc, c); break;
        }
        if (E.part) {
            const float t = warp_sum16(c, lane);
            if (!(lane & 1)) red[rq][ch * (kCols / 2) + (lane >> 1)] = t;
        }
    }
    if (E.part && do_epi) {
        __syncthreads();
        if (tid < TBN / 2) {
            const int s = n0 / 2 + tid;
            const double t = ((double)red[0][tid] + (double)red[1][tid]) + ((double)red[2][tid] + (double)red[3][tid]);
            if (s < E.nsets) E.part[(size_t)s * E.part_stride + pidx] = t;
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::kTmemCols)
                     : "memory");
}

// Persistent grouped (block-diagonal) variant: one CTA per SM walks the tile
// table (tiles c, c + grid, ...; the table is sorted by K extent) with the
// same TMA ring, MMA chain and per-chunk drain as gemm_tc_kernel.  TMEM is
// allocated once and the barrier phases run on across tiles, so the TMA and
// MMA warps start the next tile while the draining warps run this tile's
// epilogue; the epilogue's per-set sums use a named barrier of the draining
// warps only.
namespace tc {
// barrier of the draining warps only (named barrier 1)
__device__ __forceinline__ void drain_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * NDRAIN) : "memory"); }
// the same barrier, returning whether any draining thread passed true
__device__ __forceinline__ bool drain_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(32 * NDRAIN)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool failed(const int *f) { return *reinterpret_cast<const volatile int *>(f) != 0; }
}  // namespace tc

__global__ void __launch_bounds__(tc::NT, 1)
gemm_tc_grouped_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                       const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int ntn,
                       int ntiles, EpiArgs E, const GroupTile *__restrict__ gt, int *err) {
    using tc::BKF;
    using tc::kStage;
    using tc::kTileA;
    using tc::kTileB;
    using tc::STAGES;
    constexpr int TBN = tc::BN;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf[tc::GNACC], acce[tc::GNACC];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float red[4][TBN / 2];
    __shared__ float2 s_ang[2][TBN / 2];  // per-set angles of a tile, by tile parity
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_base)),
                     "r"(tc::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int st = 0; st < STAGES; st++) {
            tc::mbar_init(tc::su32(&full[st]), 1);
            tc::mbar_init(tc::su32(&empty[st]), 1);
        }
        for (int b = 0; b < tc::GNACC; b++) {
            tc::mbar_init(tc::su32(&accf[b]), 1);
            tc::mbar_init(tc::su32(&acce[b]), tc::NDRAIN);
        }
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    int issued = 0;  // producer: chunks whose loads were started

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            for (int tile = blockIdx.x; tile < ntiles && !tc::failed(&s_fail); tile += gridDim.x) {
                const GroupTile G = gt[tile / ntn];
                const int n0 = (tile % ntn) * TBN, nk = G.kext / BKF;
                for (int kb = 0; kb < nk; kb++, g++) {
                    const int st = g % STAGES;
                    if (g >= STAGES && !tc::mbar_wait(tc::su32(&empty[st]), ((g / STAGES) & 1) ^ 1)) {
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    const uint32_t base = tc::su32(smem + st * kStage);
                    const uint32_t fb = tc::su32(&full[st]);
                    tc::mbar_expect(fb, kStage);
                    const int kx = kb * BKF;
                    tc::tma_2d(base, &tmAh, kx, G.a_row, fb);
                    tc::tma_2d(base + kTileA, &tmAl, kx, G.a_row, fb);
                    tc::tma_2d(base + 2 * kTileA, &tmBh, G.k_off + kx, n0, fb);
                    tc::tma_2d(base + 2 * kTileA + kTileB, &tmBl, G.k_off + kx, n0, fb);
                    issued = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, a = 0;  // chunks (stages), accumulator groups
            for (int tile = blockIdx.x; tile < ntiles && !tc::failed(&s_fail); tile += gridDim.x) {
                const int nk = gt[tile / ntn].kext / BKF;
                for (int kb = 0; kb < nk; kb++, g++) {
                    const int st = g % STAGES, b = a % tc::GNACC;
                    const bool first = kb % tc::DGRP == 0, last = kb % tc::DGRP == tc::DGRP - 1 || kb == nk - 1;
                    if (first && a >= tc::GNACC && !tc::mbar_wait(tc::su32(&acce[b]), ((a / tc::GNACC) & 1) ^ 1)) {
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    if (!tc::mbar_wait(tc::su32(&full[st]), (g / STAGES) & 1)) {
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    tc::fence_after();
                    const uint32_t base = tc::su32(smem + st * kStage);
                    const uint32_t d = tmem + (uint32_t)(b * 2 * TBN), dc = d + (uint32_t)TBN;
#pragma unroll
                    for (int kk = 0; kk < BKF / 8; kk++) {
                        const uint64_t ah = tc::sdesc(base + kk * 32), al = tc::sdesc(base + kTileA + kk * 32);
                        const uint64_t bh = tc::sdesc(base + 2 * kTileA + kk * 32),
                                       bl = tc::sdesc(base + 2 * kTileA + kTileB + kk * 32);
                        const uint32_t accum = (first && kk == 0) ? 0u : 1u;
                        tc::mma_tf32(dc, al, bh, tc::kIdesc, accum);
                        tc::mma_tf32(dc, ah, bl, tc::kIdesc, 1u);
                        tc::mma_tf32(d, ah, bh, tc::kIdesc, accum);
                    }
                    tc::mma_commit(tc::su32(&empty[st]));
                    if (last) {
                        tc::mma_commit(tc::su32(&accf[b]));
                        a++;
                    }
                }
            }
        }
    } else {
        // draining warps: warp w reads accumulator rows (TMEM lanes) 32 (w % 4) ..
        // and columns kCols * ch .. (ch = which of the quarter's warps)
        constexpr int kCols = TBN / (tc::NDRAIN / 4);
        static_assert(kCols == 32, "the epilogue takes 16 sets per thread");
        const uint32_t lrow = (uint32_t)((warp & 3) * 32) << 16;
        const int ch = (warp - 2) >> 2, rq = warp & 3, dt = tid - 64;
        int a = 0, par = 0;  // accumulator groups drained, tile parity
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, par ^= 1) {
            const GroupTile G = gt[tile / ntn];
            const int n0 = (tile % ntn) * TBN, nk = G.kext / BKF;
            // this tile's angles; the buffer was last read two tiles ago, before
            // the draining warps' barrier of the previous tile
            if (dt < TBN / 2 && n0 / 2 + dt < E.nsets && E.kind != EPI_STORE && E.kind != EPI_FWD_LAST)
                s_ang[par][dt] = epi_angle(E, n0 / 2 + dt);
            float acc[kCols];
#pragma unroll
            for (int c = 0; c < kCols; c++) acc[c] = 0.f;
            bool ok = !tc::failed(&s_fail);
            for (int j = 0; j < (nk + tc::DGRP - 1) / tc::DGRP && ok; j++, a++) {
                const int b = a % tc::GNACC;
                if (!tc::mbar_wait(tc::su32(&accf[b]), (a / tc::GNACC) & 1)) {
                    atomicExch(&s_fail, 1);
                    ok = false;
                    break;
                }
                tc::fence_after();
#pragma unroll
                for (int q = 0; q < kCols / 16; q++) {  // 16 columns of the pair at a time
                    uint32_t r[16], rc[16];
                    const uint32_t col = tmem + lrow + (uint32_t)(b * 2 * TBN + ch * kCols + 16 * q);
                    tc::tmem_ld16(col, r);
                    tc::tmem_ld16(col + TBN, rc);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; i++) acc[16 * q + i] += __uint_as_float(r[i]) + __uint_as_float(rc[i]);
                }
                tc::fence_before();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(tc::su32(&acce[b]));
            }
            // the draining warps agree on whether the tile completed
            if (tc::drain_sync_or(!ok || tc::failed(&s_fail))) break;
            const int m = G.out_row + rq * 32 + lane;
            const int s0 = n0 / 2 + ch * (kCols / 2);  // first of this thread's sets
            const int nq = m < G.row_end ? min(kCols / 2, E.nsets - s0) : 0;
            const float2 *ang = &s_ang[par][ch * (kCols / 2)];
            float c[kCols / 2];
            switch (E.kind) {
            case EPI_STORE: epi_row16<EPI_STORE>(E, m, s0, nq, ang, acc, c); break;
            case EPI_FWD_EIG: epi_row16<EPI_FWD_EIG>(E, m, s0, nq, ang, acc, c); break;
            case EPI_FWD_PHASE: epi_row16<EPI_FWD_PHASE>(E, m, s0, nq, ang, acc, c); break;
            case EPI_FWD_LAST: epi_row16<EPI_FWD_LAST>(E, m, s0, nq, ang, acc, c); break;
            case EPI_BWD_EIG: epi_row16<EPI_BWD_EIG>(E, m, s0, nq, ang, acc, c); break;
            default: epi_row16<EPI_BWD_PHASE>(E, m, s0, nq, ang, acc, c); break;
            }
            if (E.part) {
                const float t = warp_sum16(c, lane);
                if (!(lane & 1)) red[rq][ch * (kCols / 2) + (lane >> 1)] = t;
            }
            if (E.part) {
                tc::drain_sync();
                if (dt < TBN / 2) {
                    const int s = n0 / 2 + dt;
                    const double t =
                        ((double)red[0][dt] + (double)red[1][dt]) + ((double)red[2][dt] + (double)red[3][dt]);
                    if (s < E.nsets) E.part[(size_t)s * E.part_stride + G.part_idx] = t;
                }
                tc::drain_sync();  // red is free for the next tile
            }
        }
    }
    __syncwarp();
    const bool failed = __syncthreads_or(s_fail) != 0;
    if (failed) {
        if (tid == 0) atomicOr(err, DERR_TIMEOUT);
        // let started loads land before the block exits
        if (warp == 0 && lane == 0)
            for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; kb++)
                tc::mbar_wait(tc::su32(&full[kb % STAGES]), (kb / STAGES) & 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tc::kTmemCols)
                     : "memory");
}

// Initial state of every set with the first phase separator applied:
// X = e^{-i g_1 C} psi_0 (psi_0 uniform 1/sqrt(D) or a user complex64 state);
// also keeps psi_0 as checkpoint 0.
__global__ void eig_init_kernel(float *X, float *X_lo, float *ck0, int D, int ld, int nsets, const void *cost,
                                int cost_dtype, const RoundCoef *coef, int coef_stride, const float2 *init,
                                float amp0) {
    const int s = blockIdx.y;
    if (s >= nsets) return;
    const RoundCoef cf = coef[s * coef_stride];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) {
        const float2 v = init ? init[j] : make_float2(amp0, 0.f);
        const float C = cost_dtype == 0 ? reinterpret_cast<const float *>(cost)[j]
                                        : (float)reinterpret_cast<const unsigned char *>(cost)[j];
        const float2 w = cmul(v, turn_phase(cf.g_hi, cf.g_lo, C, 0.f));
        const size_t o = (size_t)(2 * s) * ld + j;
        put(X, X_lo, o, w.x);
        put(X, X_lo, o + ld, w.y);
        if (ck0) {
            ck0[o] = v.x;
            ck0[o + ld] = v.y;
        }
    }
}

// Mean of the D cost values in a fixed order (one block): the shift c0 of the
// adjoint sweep.  Any constant gives the same gradient, because
// <mu_k|phi_k> = <lambda_p|psi_p> = <C> is real; the mean removes the
// component of lambda_p along psi_p that would otherwise dominate it.
__global__ void __launch_bounds__(256) cost_mean_kernel(const void *cost, int cost_dtype, int D, double *out) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int j = threadIdx.x; j < D; j += 256)
        acc += cost_dtype == 0 ? (double)reinterpret_cast<const float *>(cost)[j]
                               : (double)reinterpret_cast<const unsigned char *>(cost)[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w];
        *out = t / (double)D;
    }
}

// ------------------------------------------------------------ orbit kernel
// The per-orbit change of basis of the block-diagonal XY mixers: momentum
// coefficients (the products' basis) <-> amplitudes of the orbit's member
// states (the computational basis, where the cost is diagonal).  With T the
// orthogonal map from momentum coefficients to amplitudes, T restricted to a
// period-r orbit is the r x r matrix M_r[j][a] (member j, vector a).  One
// thread takes one orbit of one angle set (both the Re and Im rows); consecutive
// threads take consecutive orbits, whose vectors sit at consecutive positions of
// each block.  Round-boundary work in between (see OrbitMode):
//   INIT : X = T^T (e^{-i g_0 C} psi_0); checkpoint T^T psi_0
//   PHASE: X = T^T (e^{-i g C} T Z)
//   LAST : <C> partial sum_j C |a_j|^2 of a = T Z; L = T^T ((C - c0) a)
//   BWD  : mu = T W, phi = e^{-i g C} T P; gamma partial
//          sum_j (C_j - c0) Im(conj(mu_j) phi_j); L = T^T (e^{+i g C} mu)
// Partial sums: fixed-order block sums, float64 across warps.
template <int MODE, int RMAX>
__global__ void __launch_bounds__(kOrbitThreads) orbit_kernel(OrbitTabs T, OrbitArgs A) {
    __shared__ double red[kOrbitThreads / 32];
    // every M_r of the layout (sum of r^2 over the periods, at most
    // kOrbitSmem floats), read by all threads at once: shared-memory broadcasts
    __shared__ __align__(16) float s_mr[kOrbitSmem];
    // the full-period matrix M_RMAX and its transpose, 16-byte aligned, so
    // that both transforms read four consecutive entries at once
    constexpr int kF = RMAX <= 16 ? RMAX : 1;
    __shared__ __align__(16) float s_mf[kF * kF];
    __shared__ __align__(16) float s_mft[kF * kF];
    for (int i = threadIdx.x; i < T.mr_len; i += kOrbitThreads) s_mr[i] = T.mr[i];
    const int off_full = RMAX <= 16 ? T.mr_off[RMAX] : -1;
    if (off_full >= 0)
        for (int i = threadIdx.x; i < kF * kF; i += kOrbitThreads) {
            const float m = T.mr[off_full + i];
            s_mf[i] = m;
            s_mft[(i % kF) * kF + i / kF] = m;
        }
    __syncthreads();
    // Two adjacent lanes per (orbit, set): part 0 holds the real rows, part 1
    // the imaginary ones.  M_r is real, so each row transforms on its own;
    // the phase and the gamma term take the partner's values by a shuffle.
    const int part = threadIdx.x & 1;
    const unsigned pair_mask = 3u << ((threadIdx.x & 31) & ~1);
    const int o = blockIdx.x * kOrbitsPerBlock + (threadIdx.x >> 1);
    const int s = blockIdx.y;
    float contrib = 0.f;
    if (o < T.n_orbits && s < A.nsets) {  // the same for both lanes of a pair
        const int s0 = T.orb_start[o], r = T.orb_start[o + 1] - s0;
        const RoundCoef cf = A.coef[s * A.coef_stride + A.round];
        const size_t row = (size_t)(2 * s + part) * A.ldp;
        // (re, im) of a member from this lane's part and the partner's
        auto pair_of = [&](float v) -> float2 {
            const float w = __shfl_xor_sync(pair_mask, v, 1);
            return part ? make_float2(w, v) : make_float2(v, w);
        };
        auto take = [&](float2 z) -> float { return part ? z.y : z.x; };
        // Full-period orbits (all but a few; they come first in orbit order)
        // take a copy of the body with the period known at compile time: no
        // bound tests, M_r rows read as float4.  The sums run over the same
        // index order in both copies, so the results agree bit for bit.
        auto body = [&](auto full_tag) {
            constexpr bool FULL = decltype(full_tag)::value;
            const int R = FULL ? RMAX : r;
            const float *M = FULL ? s_mf : s_mr + T.mr_off[r];
            float c[RMAX];
            // full-period orbits start on a multiple of 16 members: their vector
            // positions and member indices are read once, 16 bytes at a time
            int pos[FULL ? RMAX : 1], mem[FULL ? RMAX : 1];
            if constexpr (FULL) {
                const int4 *vp = reinterpret_cast<const int4 *>(T.vec_pos + s0);
                const int4 *mp = reinterpret_cast<const int4 *>(T.members + s0);
#pragma unroll
                for (int q = 0; q < RMAX / 4; q++) {
                    const int4 v = __ldg(vp + q), w = __ldg(mp + q);
                    pos[4 * q] = v.x;
                    pos[4 * q + 1] = v.y;
                    pos[4 * q + 2] = v.z;
                    pos[4 * q + 3] = v.w;
                    mem[4 * q] = w.x;
                    mem[4 * q + 1] = w.y;
                    mem[4 * q + 2] = w.z;
                    mem[4 * q + 3] = w.w;
                }
            }
            auto vpos = [&](int a) -> int {
                if constexpr (FULL) return pos[a];
                else return T.vec_pos[s0 + a];
            };
            auto cost_of = [&](int j) -> float {
                int idx;
                if constexpr (FULL) idx = mem[j];
                else idx = T.members[s0 + j];
                return A.cost_dtype == 0 ? __ldg(reinterpret_cast<const float *>(A.cost) + idx)
                                         : (float)__ldg(reinterpret_cast<const unsigned char *>(A.cost) + idx);
            };
            // x = T c for this lane's row of the orbit's coefficients in `in`
            auto to_amp = [&](const float *in, float (&x)[RMAX]) {
#pragma unroll
                for (int a = 0; a < RMAX; a++)
                    if (a < R) c[a] = in[row + vpos(a)];
                // member sums accumulated side by side (independent FMA chains)
#pragma unroll
                for (int j = 0; j < RMAX; j++) x[j] = 0.f;
#pragma unroll
                for (int a = 0; a < RMAX; a++) {
                    if (a >= R) continue;
                    if constexpr (FULL) {  // row a of M^T: M[j][a], j = 4q .. 4q + 3
                        const float4 *MT4 = reinterpret_cast<const float4 *>(s_mft) + a * (RMAX / 4);
#pragma unroll
                        for (int q = 0; q < RMAX / 4; q++) {
                            const float4 m = MT4[q];
                            x[4 * q] = fmaf(m.x, c[a], x[4 * q]);
                            x[4 * q + 1] = fmaf(m.y, c[a], x[4 * q + 1]);
                            x[4 * q + 2] = fmaf(m.z, c[a], x[4 * q + 2]);
                            x[4 * q + 3] = fmaf(m.w, c[a], x[4 * q + 3]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < RMAX; j++) {
                            if (j >= R) continue;
                            x[j] = fmaf(M[j * R + a], c[a], x[j]);
                        }
                    }
                }
            };
            // c = T^T x written to this lane's row of `out` (tf32 split when out_lo)
            auto from_amp = [&](const float (&x)[RMAX], float *out, float *out_lo) {
#pragma unroll
                for (int a = 0; a < RMAX; a++) c[a] = 0.f;
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    if constexpr (FULL) {
                        const float4 *M4 = reinterpret_cast<const float4 *>(M) + j * (RMAX / 4);
#pragma unroll
                        for (int q = 0; q < RMAX / 4; q++) {
                            const float4 m = M4[q];
                            c[4 * q] = fmaf(m.x, x[j], c[4 * q]);
                            c[4 * q + 1] = fmaf(m.y, x[j], c[4 * q + 1]);
                            c[4 * q + 2] = fmaf(m.z, x[j], c[4 * q + 2]);
                            c[4 * q + 3] = fmaf(m.w, x[j], c[4 * q + 3]);
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < RMAX; a++) {
                            if (a >= R) continue;
                            c[a] = fmaf(M[j * R + a], x[j], c[a]);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < RMAX; a++) {
                    if (a >= R) continue;
                    put(out, out_lo, row + vpos(a), c[a]);
                }
            };
            float x[RMAX];
            if (MODE == ORB_INIT) {
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    int mj;
                    if constexpr (FULL) mj = mem[j];
                    else mj = T.members[s0 + j];
                    const float2 v = A.init ? A.init[mj] : make_float2(A.amp0, 0.f);
                    x[j] = part ? v.y : v.x;
                }
                if (A.ckpt) from_amp(x, A.ckpt, nullptr);
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    x[j] = take(cmul(pair_of(x[j]), turn_phase(cf.g_hi, cf.g_lo, cost_of(j), 0.f)));
                }
                from_amp(x, A.out, A.out_lo);
            } else if (MODE == ORB_PHASE) {
                to_amp(A.in, x);
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    x[j] = take(cmul(pair_of(x[j]), turn_phase(cf.g_hi, cf.g_lo, cost_of(j), 0.f)));
                }
                from_amp(x, A.out, A.out_lo);
            } else if (MODE == ORB_LAST) {
                to_amp(A.in, x);
                const float c0 = A.c0 ? (float)__ldg(A.c0) : 0.f;
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    const float C = cost_of(j);
                    contrib = fmaf(C, x[j] * x[j], contrib);  // C |x|^2 over the two lanes
                    x[j] *= C - c0;
                }
                if (A.out) from_amp(x, A.out, A.out_lo);
            } else {  // ORB_BWD
                // two matrices to read: start the second one's lines toward L2
                // while the first is fetched and transformed
#pragma unroll
                for (int a = 0; a < RMAX; a++) {
                    if (a >= R) continue;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(A.in + row + vpos(a)));
                }
                float pv[RMAX];
                to_amp(A.in_psi, pv);
                to_amp(A.in, x);
                const float c0 = A.c0 ? (float)__ldg(A.c0) : 0.f;
#pragma unroll
                for (int j = 0; j < RMAX; j++) {
                    if (j >= R) continue;
                    const float C = cost_of(j);
                    const float2 ph = turn_phase(cf.g_hi, cf.g_lo, C, 0.f);
                    const float2 phi = cmul(pair_of(pv[j]), ph);
                    const float2 mu = pair_of(x[j]);
                    if (part == 0) contrib = fmaf(C - c0, mu.x * phi.y - mu.y * phi.x, contrib);
                    // undo the phase on mu: mu conj(ph)
                    x[j] = take(make_float2(fmaf(mu.x, ph.x, mu.y * ph.y), fmaf(mu.y, ph.x, -mu.x * ph.y)));
                }
                if (A.out) from_amp(x, A.out, A.out_lo);
            }
        };
        // (the 32-wide copy would not fit the registers next to the generic one)
        if constexpr (RMAX <= 16) {
            if (r == RMAX && off_full >= 0 && (s0 & 3) == 0) body(std::integral_constant<bool, true>());
            else body(std::integral_constant<bool, false>());
        } else {
            body(std::integral_constant<bool, false>());
        }
    }
    if (MODE == ORB_LAST || MODE == ORB_BWD) {
        if (!A.part) return;  // uniform over the launch
        float v = contrib;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
        __syncthreads();
        if (threadIdx.x == 0 && s < A.nsets) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kOrbitThreads / 32; w++) t += red[w];
            A.part[(size_t)s * A.part_stride + blockIdx.x] = t;
        }
    }
}

// Block eigenvector matrices V_b (back to back, D_b x D_b row-major) into the
// stacked, zero-padded operand planes: row block_pos[b] + i of Vp is row i of
// V_b (A = V_b), of Vtp column i (A = V_b^T); eigenvalues to padded positions.
__global__ void sym_prepare_kernel(const float *V, const double *lam, const int *bdim, const int *boff,
                                   const int *bpos, int nb, int pmax, float *Vp, float *Vtp, float *Vp_lo,
                                   float *Vtp_lo, float *lam_hi, float *lam_lo) {
    const int b = blockIdx.y;
    if (b >= nb) return;
    const int Db = bdim[b], P = bpos[b + 1] - bpos[b];
    const float *Vb = V + (size_t)0;
    // offset of V_b: sum of D_b'^2 over earlier blocks
    size_t vo = 0;
    for (int q = 0; q < b; q++) vo += (size_t)bdim[q] * bdim[q];
    Vb += vo;
    const int64_t total = (int64_t)P * pmax;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / pmax), c = (int)(e % pmax);
        const size_t o = (size_t)(bpos[b] + i) * pmax + c;
        const bool in = i < Db && c < Db;
        put(Vp, Vp_lo, o, in ? Vb[(size_t)i * Db + c] : 0.f);
        put(Vtp, Vtp_lo, o, in ? Vb[(size_t)c * Db + i] : 0.f);
        if (c == 0) {
            const double l = i < Db ? lam[boff[b] + i] : 0.0;
            const float hi = (float)l;
            lam_hi[bpos[b] + i] = hi;
            lam_lo[bpos[b] + i] = (float)(l - (double)hi);
        }
    }
}

// Padded copies of V (row-major D x D) and V^T, and lambda split into two floats.
__global__ void eig_prepare_kernel(const float *V, int D, int ld, float *Vp, float *Vtp, float *Vp_lo,
                                   float *Vtp_lo, const double *lam, float *lam_hi, float *lam_lo) {
    const int64_t total = (int64_t)ld * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), c = (int)(e % ld);
        const float v = (r < D && c < D) ? V[(int64_t)r * D + c] : 0.f;
        put(Vp, Vp_lo, e, v);
        put(Vtp, Vtp_lo, (int64_t)c * ld + r, v);
        if (r == 0) {
            const double l = c < D ? lam[c] : 0.0;
            const float hi = (float)l;
            lam_hi[c] = hi;
            lam_lo[c] = (float)(l - (double)hi);
        }
    }
}

}  // namespace

cudaError_t launch_sym_prepare(const float *V, const double *lam, const int *d_bdim, const int *d_boff,
                               const int *d_bpos, int nb, int pmax, float *Vp, float *Vtp, float *Vp_lo, float *Vtp_lo,
                               float *lam_hi, float *lam_lo, cudaStream_t s) {
    dim3 grid(152, nb);
    sym_prepare_kernel<<<grid, 256, 0, s>>>(V, lam, d_bdim, d_boff, d_bpos, nb, pmax, Vp, Vtp, Vp_lo, Vtp_lo,
                                            lam_hi, lam_lo);
    return cudaGetLastError();
}

cudaError_t launch_eig_prepare(const float *V, int D, int ld, float *Vp, float *Vtp, float *Vp_lo, float *Vtp_lo,
                               const double *lam, float *lam_hi, float *lam_lo, cudaStream_t s) {
    eig_prepare_kernel<<<152 * 16, 256, 0, s>>>(V, D, ld, Vp, Vtp, Vp_lo, Vtp_lo, lam, lam_hi, lam_lo);
    return cudaGetLastError();
}

cudaError_t launch_orbit(const OrbitTabs &T, const OrbitArgs &A, cudaStream_t s) {
    if (T.max_r < 1 || T.max_r > kSymMaxN || T.mr_len < 1 || T.mr_len > kOrbitSmem) return cudaErrorInvalidValue;
    dim3 grid((T.n_orbits + kOrbitsPerBlock - 1) / kOrbitsPerBlock, A.nsets);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    // the longest orbit sets the register arrays: 16 or 32 members
    const bool r16 = T.max_r <= 16;
    switch (A.mode) {
    case ORB_INIT:
        if (r16) orbit_kernel<ORB_INIT, 16><<<grid, kOrbitThreads, 0, s>>>(T, A);
        else orbit_kernel<ORB_INIT, 32><<<grid, kOrbitThreads, 0, s>>>(T, A);
        break;
    case ORB_PHASE:
        if (r16) orbit_kernel<ORB_PHASE, 16><<<grid, kOrbitThreads, 0, s>>>(T, A);
        else orbit_kernel<ORB_PHASE, 32><<<grid, kOrbitThreads, 0, s>>>(T, A);
        break;
    case ORB_LAST:
        if (r16) orbit_kernel<ORB_LAST, 16><<<grid, kOrbitThreads, 0, s>>>(T, A);
        else orbit_kernel<ORB_LAST, 32><<<grid, kOrbitThreads, 0, s>>>(T, A);
        break;
    case ORB_BWD:
        if (r16) orbit_kernel<ORB_BWD, 16><<<grid, kOrbitThreads, 0, s>>>(T, A);
        else orbit_kernel<ORB_BWD, 32><<<grid, kOrbitThreads, 0, s>>>(T, A);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_cost_mean(const void *cost, int cost_dtype, int D, double *out, cudaStream_t s) {
    cost_mean_kernel<<<1, 256, 0, s>>>(cost, cost_dtype, D, out);
    return cudaGetLastError();
}

cudaError_t launch_eig_init(float *X, float *X_lo, float *ck0, int D, int ld, int nsets, const void *cost,
                            int cost_dtype, const RoundCoef *coef, int coef_stride, const float2 *init, float amp0,
                            cudaStream_t s) {
    dim3 grid((D + 255) / 256, nsets);
    eig_init_kernel<<<grid, 256, 0, s>>>(X, X_lo, ck0, D, ld, nsets, cost, cost_dtype, coef, coef_stride, init,
                                         amp0);
    return cudaGetLastError();
}

namespace {
EpiArgs to_args(const EigEpiParams &P) {
    EpiArgs E;
    E.kind = P.kind;
    E.M = P.M;
    E.ld = P.ld;
    E.nsets = P.nsets;
    E.out = P.out;
    E.out2 = P.out2;
    E.ckpt = P.ckpt;
    E.ck_in = P.ck_in;
    E.lam_hi = P.lam_hi;
    E.lam_lo = P.lam_lo;
    E.cost = P.cost;
    E.cost_dtype = P.cost_dtype;
    E.coef = P.coef;
    E.coef_stride = P.coef_stride;
    E.round = P.round;
    E.part = P.part;
    E.part_stride = P.part_stride;
    E.out_lo = P.out_lo;
    E.out2_lo = P.out2_lo;
    E.c0 = P.c0;
    return E;
}
}  // namespace

cudaError_t launch_eig_gemm_simt(const float *A, const float *B, int Mp, int Np, int Kp, const EigEpiParams &P,
                                 cudaStream_t s) {
    dim3 grid(Mp / BM, Np / BN);
    gemm_simt_kernel<<<grid, NT, 0, s>>>(A, B, Kp, Kp, Kp, to_args(P), nullptr);
    return cudaGetLastError();
}

int eig_split_max_tail() {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

cudaError_t launch_eig_gemm_tc(const CUtensorMap &a_hi, const CUtensorMap &a_lo, const CUtensorMap &b_hi,
                               const CUtensorMap &b_lo, int Mp, int Np, int Kp, const EigEpiParams &P, float *d_ws,
                               unsigned *d_cnt, int *err, cudaStream_t s) {
    static int attr_done[kMaxDevices];
    {
        cudaError_t e = smem_attr_once(gemm_tc_kernel, (int)tc::kSmem, attr_done);
        if (e != cudaSuccess) return e;
    }
    const int ntn = Np / tc::BN;
    const int tiles = (Mp / tc::BM) * ntn;
    // One block per SM: with W whole waves and R < nsm tiles left over, the
    // R tiles run as S K-segments each when that ends sooner, W + ceil(R S /
    // nsm) / S waves against W + 1 (S = 2..kMaxSeg).
    const int nsm = eig_split_max_tail();
    SplitArgs sp{tiles, 1, d_ws, d_cnt};
    const int W = tiles / nsm, R = tiles - W * nsm;
    if (d_ws && d_cnt && W >= 1 && R > 0 && R <= eig_split_max_tail()) {
        double best = 1.0;  // the unsplit tail: one more wave
        for (int S = 2; S <= kEigMaxSeg; S++) {
            const double t = (double)((R * S + nsm - 1) / nsm) / S;
            if (t < best - 1e-9 && Kp / tc::BKF >= 8 * S) {
                best = t;
                sp.nseg = S;
            }
        }
        if (sp.nseg > 1) sp.full = W * nsm;
    }
    const int grid = sp.full + (tiles - sp.full) * sp.nseg;
    gemm_tc_kernel<<<grid, tc::NT, tc::kSmem, s>>>(a_hi, a_lo, b_hi, b_lo, Kp, ntn, to_args(P), sp, err, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_eig_gemm_simt_grouped(const float *A, int lda, const float *B, int ldb, int Np,
                                         const GroupTile *d_tiles, int n_mtiles, const EigEpiParams &P,
                                         cudaStream_t s) {
    if (n_mtiles <= 0) return cudaSuccess;
    dim3 grid(n_mtiles, Np / BN);
    gemm_simt_kernel<<<grid, NT, 0, s>>>(A, B, 0, lda, ldb, to_args(P), d_tiles);
    return cudaGetLastError();
}

cudaError_t launch_eig_gemm_tc_grouped(const CUtensorMap &a_hi, const CUtensorMap &a_lo, const CUtensorMap &b_hi,
                                       const CUtensorMap &b_lo, int Np, const GroupTile *d_tiles, int n_mtiles,
                                       const EigEpiParams &P, int *err, cudaStream_t s) {
    if (n_mtiles <= 0) return cudaSuccess;
    static int attr_done[kMaxDevices];
    {
        cudaError_t e = smem_attr_once(gemm_tc_kernel, (int)tc::kSmem, attr_done);
        if (e != cudaSuccess) return e;
    }
    static int attr_done_p[kMaxDevices];
    {
        cudaError_t e = smem_attr_once(gemm_tc_grouped_kernel, (int)tc::kSmem, attr_done_p);
        if (e != cudaSuccess) return e;
    }
    const int ntn = Np / tc::BN;
    const int tiles = n_mtiles * ntn;
    const int grid = std::min(tiles, eig_split_max_tail());  // one CTA per SM
    gemm_tc_grouped_kernel<<<grid, tc::NT, tc::kSmem, s>>>(a_hi, a_lo, b_hi, b_lo, ntn, tiles, to_args(P), d_tiles,
                                                           err);
    return cudaGetLastError();
}

}  // namespace qg
