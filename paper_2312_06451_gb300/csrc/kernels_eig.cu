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
};

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
    case EPI_FWD_EIG: {  // Y = e^{-i b lambda} v, checkpoint V^T phi
        if (E.ckpt) {
            E.ckpt[o_re] = v.x;
            E.ckpt[o_im] = v.y;
        }
        const float2 w = cmul(v, turn_phase(cf.b_hi, cf.b_lo, E.lam_hi[j], E.lam_lo[j]));
        E.out[o_re] = w.x;
        E.out[o_im] = w.y;
        break;
    }
    case EPI_FWD_PHASE: {  // X = e^{-i g' C} v, checkpoint psi_k
        if (E.ckpt) {
            E.ckpt[o_re] = v.x;
            E.ckpt[o_im] = v.y;
        }
        const float2 w = cmul(v, turn_phase(cf.g_hi, cf.g_lo, cost_at(E, j), 0.f));
        E.out[o_re] = w.x;
        E.out[o_im] = w.y;
        break;
    }
    case EPI_FWD_LAST: {  // psi_p: <C> partial, store psi_p and lambda_p = C psi_p
        const float C = cost_at(E, j);
        contrib = C * fmaf(v.x, v.x, v.y * v.y);
        if (E.out) {
            E.out[o_re] = v.x;
            E.out[o_im] = v.y;
        }
        if (E.out2) {
            E.out2[o_re] = C * v.x;
            E.out2[o_im] = C * v.y;
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
        E.out[o_re] = w.x;
        E.out[o_im] = w.y;
        break;
    }
    case EPI_BWD_PHASE: {  // gamma partial with phi = e^{-i g C} psi_{k-1}, then undo the phase
        const float C = cost_at(E, j);
        const float2 ph = turn_phase(cf.g_hi, cf.g_lo, C, 0.f);
        const float2 phi = cmul(make_float2(E.ck_in[o_re], E.ck_in[o_im]), ph);
        contrib = C * (v.x * phi.y - v.y * phi.x);
        if (E.out) {
            const float2 w = make_float2(fmaf(v.x, ph.x, v.y * ph.y), fmaf(v.y, ph.x, -v.x * ph.y));
            E.out[o_re] = w.x;
            E.out[o_im] = w.y;
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
                 EpiArgs E) {
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];
    __shared__ float red[BN / 2][17];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    // global -> register staging: each thread loads 8 floats of A and of B
    const int lr = tid >> 1, lk = (tid & 1) * 8;
    const float *Ag = A + (size_t)(m0 + lr) * lda + lk;
    const float *Bg = B + (size_t)(n0 + lr) * ldb + lk;
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
    const int nk = Kp / BK;
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
        if (m >= E.M) continue;
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
            if (s < E.nsets) E.part[(size_t)s * E.part_stride + blockIdx.x] = t;
        }
    }
}

// Initial state of every set with the first phase separator applied:
// X = e^{-i g_1 C} psi_0 (psi_0 uniform 1/sqrt(D) or a user complex64 state);
// also keeps psi_0 as checkpoint 0.
__global__ void eig_init_kernel(float *X, float *ck0, int D, int ld, int nsets, const void *cost, int cost_dtype,
                                const RoundCoef *coef, int coef_stride, const float2 *init, float amp0) {
    const int s = blockIdx.y;
    if (s >= nsets) return;
    const RoundCoef cf = coef[s * coef_stride];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) {
        const float2 v = init ? init[j] : make_float2(amp0, 0.f);
        const float C = cost_dtype == 0 ? reinterpret_cast<const float *>(cost)[j]
                                        : (float)reinterpret_cast<const unsigned char *>(cost)[j];
        const float2 w = cmul(v, turn_phase(cf.g_hi, cf.g_lo, C, 0.f));
        const size_t o = (size_t)(2 * s) * ld + j;
        X[o] = w.x;
        X[o + ld] = w.y;
        if (ck0) {
            ck0[o] = v.x;
            ck0[o + ld] = v.y;
        }
    }
}

// Padded copies of V (row-major D x D) and V^T, and lambda split into two floats.
__global__ void eig_prepare_kernel(const float *V, int D, int ld, float *Vp, float *Vtp, const double *lam,
                                   float *lam_hi, float *lam_lo) {
    const int64_t total = (int64_t)ld * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / ld), c = (int)(e % ld);
        const float v = (r < D && c < D) ? V[(int64_t)r * D + c] : 0.f;
        Vp[e] = v;
        Vtp[(int64_t)c * ld + r] = v;
        if (r == 0) {
            const double l = c < D ? lam[c] : 0.0;
            const float hi = (float)l;
            lam_hi[c] = hi;
            lam_lo[c] = (float)(l - (double)hi);
        }
    }
}

}  // namespace

cudaError_t launch_eig_prepare(const float *V, int D, int ld, float *Vp, float *Vtp, const double *lam,
                               float *lam_hi, float *lam_lo, cudaStream_t s) {
    eig_prepare_kernel<<<152 * 16, 256, 0, s>>>(V, D, ld, Vp, Vtp, lam, lam_hi, lam_lo);
    return cudaGetLastError();
}

cudaError_t launch_eig_init(float *X, float *ck0, int D, int ld, int nsets, const void *cost, int cost_dtype,
                            const RoundCoef *coef, int coef_stride, const float2 *init, float amp0,
                            cudaStream_t s) {
    dim3 grid((D + 255) / 256, nsets);
    eig_init_kernel<<<grid, 256, 0, s>>>(X, ck0, D, ld, nsets, cost, cost_dtype, coef, coef_stride, init, amp0);
    return cudaGetLastError();
}

cudaError_t launch_eig_gemm_simt(const float *A, const float *B, int Mp, int Np, int Kp, const EigEpiParams &P,
                                 cudaStream_t s) {
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
    dim3 grid(Mp / BM, Np / BN);
    gemm_simt_kernel<<<grid, NT, 0, s>>>(A, B, Kp, Kp, Kp, E);
    return cudaGetLastError();
}

}  // namespace qg
