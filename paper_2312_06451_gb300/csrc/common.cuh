// Internal declarations shared by the library's CUDA translation units.
// Not part of the public ABI (that is include/qaoa.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace qg {

// ---------------------------------------------------------------- errors
// Bits of the device error word (ctx->d_err); kernels set them with atomicOr
// instead of trapping, the host reads the word after a synchronising call.
enum DevErr : int {
    DERR_BAD_DESC = 1,   // a block found no launch descriptor for its index
    DERR_BAD_ANGLE = 2,  // a non-finite angle reached the coefficient kernel
    DERR_BAD_COST = 4,   // a u8 cost above the phase-table size
};

// ------------------------------------------------- per-round coefficients
// Produced on the device from the float64 angles (prep kernel), consumed by
// every mixer/phase kernel.  The X rotation e^{-i b X} = cos b - i sin b X is
// applied in factored form: with |tan b| <= 1 it is cos b * (1 - i tan b X)
// (bmode 0, bt = tan b, bs = cos b); otherwise sin b * (cot b - i X) (bmode 1,
// bt = cot b, bs = sin b).  The scalar factor is applied once per pass.
struct RoundCoef {
    float bt;
    float bs;
    int bmode;
    float g_hi;  // gamma / (2 pi), float32 head
    float g_lo;  // gamma / (2 pi) - g_hi, float32 tail
    float cb;    // cos b
    float sb;    // sin b
    float pad;
};

// Phase table entries per (unit, round) for uint8 costs: T[c] = e^{-i gamma c}.
constexpr int kPhaseTable = 256;

// -------------------------------------------------- pass descriptors (X)
enum PassFlags : uint32_t {
    PF_PHASE = 1u,       // fwd: e^{-i g C} before the rotations; bwd: gamma
                         //      partial and e^{+i g C} after the rotations
    PF_E = 2u,           // fwd: expectation partial after the rotations
    PF_LAM_FROM_C = 4u,  // bwd: lambda = C psi (first adjoint pass)
    PF_GEN_INIT = 8u,    // fwd: psi = amp0 everywhere instead of a load
    PF_UNPHASE_PSI = 16u // bwd: also undo the phase on psi (psi_out written)
};

// One pass of one unit (= one angle set of one problem).  A tile is 2^T
// amplitudes: local bit j of the tile index maps to global bit gpos[j]; the
// remaining n - T global bits (fpos, ascending) enumerate the tiles.
struct PassDesc {
    const float2 *psi_in;
    float2 *psi_out;      // nullptr: do not store psi
    const float2 *lam_in;
    float2 *lam_out;      // nullptr: do not store lambda
    const void *cost;
    const RoundCoef *coef;
    const float2 *table;  // uint8 costs: this round's phase table
    double *part_beta;    // [tile] partial sums, this pass
    double *part_gamma;   // [tile]
    double *part_E;       // [tile]
    float amp0;
    uint32_t active;      // local bits rotated in this pass
    uint32_t flags;
    uint32_t ntiles;
    uint8_t n;
    uint8_t nfree;
    uint8_t pad[2];
    uint8_t gpos[16];
    uint8_t fpos[36];
};

// Whole-state-on-chip kernel for small n (all rounds in one block).
struct SmallDesc {
    const void *cost;
    const float2 *init;
    const RoundCoef *coef;   // p entries
    const float2 *table;     // p * kPhaseTable entries (uint8 costs)
    double *E_out;
    double *grad_out;        // 2p entries or nullptr
    int n;
    int p;
    float amp0;
    int pad;
};

struct PrepDesc {
    const double *angles;  // 2p
    RoundCoef *coef;       // p
    float2 *table;         // p * kPhaseTable, or nullptr
    int p;
    int tsize;             // table entries used (<= kPhaseTable)
};

struct RedDesc {
    const double *part;  // [(2p+1)][stride]
    int64_t stride;
    int cntE, cntB, cntG;
    int p;
    double *E_out;
    double *grad_out;    // nullptr: expectation only
};

// ------------------------------------------------------- launch wrappers
// Each returns the cudaError_t of the launch.
cudaError_t launch_prep(const PrepDesc *d_descs, int ndesc, int *d_err, cudaStream_t s);
cudaError_t launch_reduce(const RedDesc *d_descs, int ndesc, cudaStream_t s);
cudaError_t launch_small(const SmallDesc *d_descs, int ndesc, int cost_dtype, int want_grad,
                         int max_n, int *d_err, cudaStream_t s);
// T: tile bits (12, 13, 14); bwd: 0 forward, 1 adjoint.
cudaError_t launch_xpass(int T, int bwd, int cost_dtype, const PassDesc *d_descs,
                         const uint32_t *d_tile_begin, int ndesc, uint32_t total_tiles,
                         int *d_err, cudaStream_t s);
bool xpass_supported(int T, int bwd);
int small_max_n();

// Cost precompute (kernels_cost.cu).
cudaError_t launch_cost_maxcut(int n, const uint64_t *nbr_hi_host, const float *d_w_edges,
                               const int32_t *d_edges, int m, int weighted, int64_t dim,
                               void *d_out, int dtype, cudaStream_t s);
cudaError_t launch_cost_sk(int n, const int32_t *d_Jq, const double *d_Jd, int exact,
                           int64_t dim, float *d_out, cudaStream_t s);
cudaError_t launch_cost_dks(int n, int k, const uint64_t *nbr_hi_host, int64_t dim, void *d_out,
                            int dtype, cudaStream_t s);
cudaError_t launch_dicke_states(int n, int k, int64_t dim, uint64_t *d_out, cudaStream_t s);
cudaError_t launch_ring_hamiltonian(int n, int k, int64_t dim, double *d_H, cudaStream_t s);
int binom_table_max();
cudaError_t upload_binom_table();

}  // namespace qg
