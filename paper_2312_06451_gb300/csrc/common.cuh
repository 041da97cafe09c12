// Internal declarations shared by the library's CUDA translation units.
// Not part of the public ABI (that is include/qaoa.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace qg {

// ---------------------------------------------------------------- errors
// Bits of the device error word (ctx->d_err); kernels set them with atomicOr
// instead of trapping, the host reads the word after a synchronising call.
enum DevErr : int {
    DERR_BAD_DESC = 1,   // a block found no launch descriptor for its index
    DERR_BAD_ANGLE = 2,  // a non-finite angle reached the coefficient kernel
    DERR_BAD_COST = 4,   // a u8 cost above the phase-table size
    DERR_TIMEOUT = 8,    // a bounded mbarrier wait gave up
};

// ------------------------------------------------- per-round coefficients
// Produced on the device from the float64 angles (prep kernel), consumed by
// every mixer/phase kernel.
//
// The pass kernels keep states in the twisted basis s_x = (-i)^{|x|} psi_x
// (a diagonal unitary: it commutes with the phase separator and leaves |psi|^2
// unchanged).  There e^{-i b X} becomes the real rotation
// [[cos b, sin b], [-sin b, cos b]] acting alike on real and imaginary parts.
// bmode 0 applies it as cos b * [[1, t], [-t, 1]], t = tan b, with the cos b
// factors applied once per stage or per pass; bmode 2 (|cos b| tiny) applies
// the rotation directly.
struct RoundCoef {
    float bt;      // tan b
    float cb;      // cos b
    float sb;      // sin b
    int bmode;     // 0: tan form, 2: direct form
    float g_hi;    // gamma / (2 pi), float32 head
    float g_lo;    // gamma / (2 pi) - g_hi, float32 tail
    int rescale;   // 1: apply the cos factors after every stage (|cos b| < 1/4)
    float b_hi;    // beta / (2 pi), float32 head (eigenbasis mixers)
    float b_lo;    // beta / (2 pi) - b_hi
    float pad;
};

// Phase table entries per (unit, round) for uint8 costs: T[c] = e^{-i gamma c}.
constexpr int kPhaseTable = 256;

// Device-side waits give up after this much wall-clock time (nanoseconds of
// the GPU's global timer); a completed copy or barrier takes microseconds.
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// -------------------------------------------------- pass descriptors (X)
enum PassFlags : uint32_t {
    PF_PHASE = 1u,       // fwd: e^{-i g C} before the rotations; bwd: gamma
                         //      partial and e^{+i g C} after the rotations
    PF_E = 2u,           // fwd: expectation partial after the rotations
    PF_LAM_FROM_C = 4u,  // bwd: lambda = C psi (first adjoint pass)
    PF_GEN_INIT = 8u,    // fwd: psi = amp0 everywhere instead of a load
    PF_UNPHASE_PSI = 16u, // bwd: also undo the phase on psi (psi_out written)
    PF_TWIST_IN = 32u,   // fwd: psi_in is a user state in the plain basis
    PF_WDIAG = 64u,      // general X mixer: fwd: e^{-i b G(|x|)} on load; bwd: its
                         // beta partial and its undo after the rotations
    PF_FUSED = 128u      // round boundary: the tile bits are the last group of round
                         // k (coef) and the first of round k+1 (coef2).  fwd: rotations
                         // of round k, e^{-i g_{k+1} C}, rotations of round k+1; bwd:
                         // undo round k+1 (beta partial -> part_beta), gamma_{k+1}
                         // partial and phase undo, undo round k (-> part_beta2)
};

// Per-warp partial sums per tile of the pass kernel.
constexpr int kPassWarps = 8;

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
    const float4 *wtab;   // PF_WDIAG: per weight w (cos, -sin of b G(w), G(w), 0)
    double *part_beta;    // [tile] partial sums, this pass
    double *part_gamma;   // [tile]
    double *part_E;       // [tile]
    const RoundCoef *coef2;  // PF_FUSED: round k+1 (coef: round k)
    double *part_beta2;      // PF_FUSED adjoint: round k's beta partials
    // TMA tensor maps (CUtensorMap, 64-byte aligned, device memory) of the
    // gathered tile of psi_in / lam_in / cost, or nullptr: then the tile is
    // fetched as 2^(T-c) one-dimensional bulk copies of 2^c elements.
    const void *tm_psi;
    const void *tm_lam;
    const void *tm_cost;
    // adjoint: the constant c0 subtracted from C wherever the adjoint uses the
    // cost as an operator (lambda_p = (C - c0) psi_p and the gamma partials);
    // nullptr = 0.  The gradient does not depend on c0; c0 = <C> keeps lambda
    // free of the large common component c0 psi.
    const double *c0;
    float amp0;
    uint32_t active;      // local bits rotated in this pass
    uint32_t flags;
    uint32_t ntiles;
    uint8_t n;
    uint8_t nfree;
    uint8_t c;            // local bits 0..c-1 are global bits 0..c-1 (one contiguous run)
    uint8_t pad;
    uint8_t gpos[16];
    uint8_t fpos[36];
};

// Tile of the pass kernel: 2^12 amplitudes, 256 threads x 16 amplitudes.
constexpr int kPassTileBits = 12;

// Whole-state-on-chip kernel for small n (all rounds in one block).
struct SmallDesc {
    const void *cost;
    const float2 *init;
    const RoundCoef *coef;   // p entries (p n for multi-angle)
    const float2 *table;     // p * kPhaseTable entries (uint8 costs)
    double *E_out;
    double *grad_out;        // 2p entries or nullptr
    int n;
    int p;
    float amp0;
    int nq;                  // multi-angle: n coefficients per round (else 0)
    const double *wts;       // general X mixer: Hadamard-basis weights d_0..d_n (else nullptr)
    const double *angles_beta;  // general X mixer: beta_1..beta_p (the unit's angles)
};

struct PrepDesc {
    const double *angles;  // p (nq or 1) betas, then p gammas
    RoundCoef *coef;       // p (nq or 1) entries; general X mixer: 2 per round
    float2 *table;         // p * kPhaseTable, or nullptr
    int p;
    int tsize;             // table entries used (<= kPhaseTable)
    int nq;                // multi-angle: one beta per qubit (n), else 0
    int gm_n;              // general X mixer: qubits n (else 0)
    const double *wts;     // general X mixer: Hadamard-basis weights d_0..d_n
    float4 *wtab;          // general X mixer: p x (n + 1) weight phases
};

// Two-level deterministic reduction of the per-(tile, warp) partial sums.
// Level 1: one block per chunk of at most kRedChunk partials -> level2[i].
// Level 2: one warp per output sums its chunks in order, times scale.
constexpr int kRedChunk = 8192;
struct RedChunk {
    const double *src;
    int cnt;
    int pad;
};
struct RedOut {
    int first;      // first chunk
    int n;          // chunks
    double *out;    // device result
    double scale;   // 1 for <C>, 2 for the derivatives (2 Im <...>)
};

// -------------------------------------------- eigenbasis mixer (kernels_eig)
enum EigEpi {
    EPI_STORE = 0,      // out = the product (block-diagonal path: the orbit kernel follows)
    EPI_FWD_EIG = 1,    // Y = e^{-i b lambda} (V^T X); checkpoint V^T phi
    EPI_FWD_PHASE = 2,  // X = e^{-i g' C} (V Y); checkpoint psi_k
    EPI_FWD_LAST = 3,   // psi_p = V Y; <C> partials; lambda_p = C psi_p
    EPI_BWD_EIG = 4,    // beta partials; undo e^{-i b lambda}
    EPI_BWD_PHASE = 5   // gamma partials; undo e^{-i g C}
};

struct EigEpiParams {
    int kind;
    int M;          // valid rows (D)
    int ld;         // padded row length
    int nsets;      // valid sets
    float *out;
    float *out2;
    float *ckpt;
    const float *ck_in;
    const float *lam_hi, *lam_lo;
    const void *cost;
    int cost_dtype;
    const RoundCoef *coef;
    int coef_stride;
    int round;
    double *part;   // [set][M tile]
    int part_stride;
    float *out_lo;  // tensor-core path: remainder planes of split outputs
    float *out2_lo;
    const double *c0;  // adjoint epilogues: cost shift (lambda_p = (C - c0) psi_p, gamma partials)
};

// Grouped products: tile i covers output rows out_row .. out_row + 127 of block
// rows valid below row_end, A rows a_row .., K columns 0 .. kext of A and
// k_off .. k_off + kext of B.
struct GroupTile {
    int a_row, k_off, kext, out_row, row_end, part_idx;
};
// Vp_lo / Vtp_lo non-null: Vp / Vtp get the tf32 heads, *_lo the remainders.
cudaError_t launch_eig_prepare(const float *V, int D, int ld, float *Vp, float *Vtp, float *Vp_lo, float *Vtp_lo,
                               const double *lam, float *lam_hi, float *lam_lo, cudaStream_t s);
// Mean of a cost vector (D entries) into *out, fixed summation order; one block.
cudaError_t launch_cost_mean(const void *cost, int cost_dtype, int D, double *out, cudaStream_t s);
cudaError_t launch_eig_init(float *X, float *X_lo, float *ck0, int D, int ld, int nsets, const void *cost,
                            int cost_dtype, const RoundCoef *coef, int coef_stride, const float2 *init, float amp0,
                            cudaStream_t s);
// out^T[Np][Mp] = A[Mp][Kp] * B[Np][Kp]^T with a fused epilogue; Mp, Np, Kp
// multiples of 128.
cudaError_t launch_eig_gemm_simt(const float *A, const float *B, int Mp, int Np, int Kp, const EigEpiParams &P,
                                 cudaStream_t s);
// Grouped (block-diagonal) variants: d_tiles holds n_mtiles GroupTile entries;
// lda / ldb are the row lengths of A and B.
cudaError_t launch_eig_gemm_simt_grouped(const float *A, int lda, const float *B, int ldb, int Np,
                                         const GroupTile *d_tiles, int n_mtiles, const EigEpiParams &P,
                                         cudaStream_t s);
cudaError_t launch_eig_gemm_tc_grouped(const CUtensorMap &a_hi, const CUtensorMap &a_lo, const CUtensorMap &b_hi,
                                       const CUtensorMap &b_lo, int Np, const GroupTile *d_tiles, int n_mtiles,
                                       const EigEpiParams &P, int *err, cudaStream_t s);
// tcgen05 3xTF32 product with the same epilogues; tensor maps (2-d, K-major,
// 32-float boxes x 128 rows, 128-byte swizzle) of the operand planes.  The
// tiles of a last, partial wave may be split along K: d_ws holds
// eig_split_max_tail() x kEigMaxSeg partial 128 x 128 float tiles and d_cnt
// eig_split_max_tail() counters, zero before the first product of a call
// (each product leaves them zero).  d_ws = nullptr: no split.
constexpr int kEigMaxSeg = 4;
int eig_split_max_tail();
cudaError_t launch_eig_gemm_tc(const CUtensorMap &a_hi, const CUtensorMap &a_lo, const CUtensorMap &b_hi,
                               const CUtensorMap &b_lo, int Mp, int Np, int Kp, const EigEpiParams &P, float *d_ws,
                               unsigned *d_cnt, int *err, cudaStream_t s);
constexpr int kEigTile = 128;   // M and N tile of the eigenbasis products
constexpr int kEigSetTile = 64; // sets per N tile

// --------------------------------------------- per-device launch settings
// Kernel attributes (the opt-in shared-memory size) belong to one device's
// context, so each device raises them for itself, the first time a launch on
// it needs them.  `done` holds one entry per device index: the size set so
// far.  Concurrent first calls both set the same value, which is harmless.
constexpr int kMaxDevices = 64;

template <typename Kern>
cudaError_t smem_attr_once(Kern kern, int bytes, int *done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (__atomic_load_n(&done[dev], __ATOMIC_ACQUIRE) >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) __atomic_store_n(&done[dev], bytes, __ATOMIC_RELEASE);
    return e;
}

// ------------------------------------------- XY-mixer cyclic symmetry (xy_sym.cu)
// Orbits of the weight-k states under the cyclic qubit shift and the real
// momentum basis that block-diagonalises the ring and clique mixers.  Vectors
// are numbered like orbit members (orbit o owns entries orb_start[o] ..
// orb_start[o+1] of members and of the vec_* arrays); vector a of a period-r
// orbit has the values M_r[j][a] = mr[mr_off[r] + j r + a] on its members.
// Positions: block b holds block_dim[b] vectors at padded positions
// block_pos[b] .. block_pos[b] + block_dim[b]; block_pos[b + 1] - block_pos[b]
// is a multiple of kSymPad.
constexpr int kSymMaxN = 32;  // longest orbit the orbit kernel holds in registers
constexpr int kSymPad = 128;  // block padding (the product tiles)
struct SymLayout {
    int n = 0, k = 0, D = 0, n_orbits = 0, ldp = 0, pmax = 0;
    std::vector<int> block_m, block_dim, block_off, block_pos;
    std::vector<int> orb_start, members, vec_pos, vec_block, vec_t, vec_sin;
    std::vector<int> orbit_of, member_of, mr_off;
    std::vector<double> mr;
};
bool build_sym_layout(int n, int k, SymLayout &L);
double sym_basis_value(int r, int t, int sin_part, int j);
// Dense block matrices Q_b^T H Q_b (row-major, block after block), mixer_kind
// 0 ring, 1 clique.
void sym_block_hamiltonians(int mixer_kind, const SymLayout &L, std::vector<double> &H);

// Device tables of a layout for the orbit kernel.
struct OrbitTabs {
    const int *orb_start;  // n_orbits + 1
    const int *members;    // Dicke index of each member
    const int *vec_pos;    // padded position of each vector
    const float *mr;       // M_r matrices (float)
    const int *mr_off;     // n + 1 offsets into mr (-1: no orbit of that period)
    int n_orbits;
    int max_r;             // longest orbit (<= kSymMaxN)
    int mr_len;            // floats in mr (<= kOrbitSmem)
};
// Shared-memory room for the M_r matrices: the sum of r^2 over the periods r
// that divide n is at most 1.34 n^2 for n <= 32.
constexpr int kOrbitSmem = 1400;
// Orbit-kernel modes (one launch per round boundary, all sets of a job).
enum OrbitMode {
    ORB_INIT = 0,   // X = T^T (e^{-i g_0 C} psi_0); ckpt = T^T psi_0
    ORB_PHASE = 1,  // X = T^T (e^{-i g_{r+1} C} T Z)
    ORB_LAST = 2,   // <C> partials of T Z; L = T^T ((C - c0) T Z)
    ORB_BWD = 3     // mu = T W, phi = e^{-i g_r C} T P; gamma partials; L = T^T (e^{+i g_r C} mu)
};
struct OrbitArgs {
    int mode;
    int D, ldp, nsets, round;
    const float *in;      // Z (PHASE, LAST) or W (BWD): [2S][ldp]
    const float *in_psi;  // BWD: checkpointed psi_{r-1} in the momentum basis
    float *out, *out_lo;  // X or L (tf32 head and remainder when out_lo)
    float *ckpt;          // INIT: T^T psi_0
    const float2 *init;   // INIT: user psi_0 (computational basis) or nullptr
    float amp0;
    const void *cost;
    int cost_dtype;
    const RoundCoef *coef;
    int coef_stride;
    const double *c0;     // LAST / BWD: cost shift
    double *part;         // LAST / BWD: [set][orbit block] partial sums
    int part_stride;
};
constexpr int kOrbitThreads = 128;                   // threads per block of the orbit kernel
constexpr int kOrbitsPerBlock = kOrbitThreads / 2;  // two threads (real, imaginary rows) per orbit
cudaError_t launch_orbit(const OrbitTabs &T, const OrbitArgs &A, cudaStream_t s);
// Padded block matrices of a symmetric eigendecomposition: A = V_b (or V_b^T)
// stacked as rows block_pos[b] .. of a [ldp][pmax] matrix (zero padded), the
// tf32 split planes when *_lo is set; eigenvalues at padded positions.
cudaError_t launch_sym_prepare(const float *V, const double *lam, const int *d_bdim, const int *d_boff,
                               const int *d_bpos, int nb, int pmax, float *Vp, float *Vtp, float *Vp_lo, float *Vtp_lo,
                               float *lam_hi, float *lam_lo, cudaStream_t s);

// ------------------------------------------------------- launch wrappers
// Each returns the cudaError_t of the launch.
cudaError_t launch_prep(const PrepDesc *d_descs, int ndesc, int *d_err, cudaStream_t s);
cudaError_t launch_reduce(const RedChunk *d_chunks, int nchunks, double *d_level2, const RedOut *d_outs,
                          int nouts, cudaStream_t s);
cudaError_t launch_small(const SmallDesc *d_descs, int ndesc, int cost_dtype, int want_grad,
                         int max_n, int *d_err, cudaStream_t s);
// bwd: 0 forward, 1 adjoint.  Persistent launch over total_tiles tiles.
// var: 0 transverse field, 1 multi-angle, 2 general X mixer (half rounds)
// d_sched: this launch's tile counter, zero when the launch starts.
// cost_free: no descriptor of the launch reads the cost vector.
// fused: every descriptor is a round-boundary pass (PF_FUSED; var 0 only).
cudaError_t launch_xpass(int bwd, int cost_dtype, int nbuf, int var, const PassDesc *d_descs,
                         const uint32_t *d_tile_begin, int ndesc, uint32_t total_tiles,
                         int *d_err, uint32_t *d_sched, int cost_free, int fused, cudaStream_t s);
int small_max_n();
// n = 12, transverse-field mixer: one CTA per angle set keeps the whole state
// as one register-staged tile (descriptors as for launch_small).
cudaError_t launch_tile12(const SmallDesc *d_descs, int ndesc, int cost_dtype, int want_grad, int *d_err,
                          cudaStream_t s);
// Diagnostic: a bounded wait on a barrier nothing completes (sets DERR_TIMEOUT).
cudaError_t launch_wait_probe(int *d_err, cudaStream_t s);

// Cost precompute (kernels_cost.cu).
cudaError_t launch_cost_maxcut(int n, const uint64_t *nbr_hi_host, const float *d_w_edges,
                               const int32_t *d_edges, int m, int weighted, int64_t dim,
                               void *d_out, int dtype, cudaStream_t s);
cudaError_t launch_cost_sk(int n, const int32_t *d_Jq, const double *d_Jd, int exact,
                           int64_t dim, float *d_out, cudaStream_t s);
cudaError_t launch_cost_dks(int n, int k, const uint64_t *nbr_hi, int64_t dim, void *d_out, int dtype,
                            int kvc, int m, cudaStream_t s);
cudaError_t launch_dicke_states(int n, int k, int64_t dim, uint64_t *d_out, cudaStream_t s);
cudaError_t launch_ring_hamiltonian(int n, int k, int64_t dim, double *d_H, cudaStream_t s);
cudaError_t launch_clique_hamiltonian(int n, int k, int64_t dim, double *d_H, cudaStream_t s);

// Grover mixer as a rank-one update on a stored state vector (kernels_rank1.cu).
enum R1Mode { R1_FWD = 0, R1_LAST = 1, R1_BWD = 2 };
enum R1ScalarMode { R1_SFWD = 0, R1_SLAST = 1, R1_SBWD = 2 };
struct R1Desc {
    const void *cost;
    const float2 *init;     // user psi_0 (16-byte aligned) or nullptr: amp0 everywhere
    const RoundCoef *coef;  // p entries (the round's gamma as g_hi + g_lo)
    const float2 *table;    // uint8 costs: p * kPhaseTable entries e^{-i gamma_r c}
    const double *angles;   // beta_0..beta_{p-1}, gamma_0..gamma_{p-1}
    float2 *phi;            // ckpt: phi_0..phi_{p-1} at stride ld; else one vector
    float2 *lam;            // gradient runs: the adjoint vector
    double *part;           // [slot][3] per-block sums (min(tiles, grid) slots)
    double *scal;           // 4 p + 3 scalars (layout in kernels_rank1.cu)
    double *E;
    double *grad;           // 2p, or nullptr
    int64_t dim;
    int64_t ld;             // vector stride (even, >= dim)
    int p;
    int ckpt;
    float amp0;
    int pad;
};
int r1_tile_amps();
uint32_t r1_max_grid();                       // upper bound of r1_grid over modes
uint32_t r1_grid(int mode, int cost_dtype);   // blocks of one pass kernel (persistent: a multiple of the SMs)
// grid: blocks of the pass (the same value for every pass and scalar launch
// over one descriptor list: it fixes the slot layout of the partials).
// err: the device error word (DERR_TIMEOUT when a bounded copy wait gives up).
cudaError_t launch_r1_pass(int mode, int cost_dtype, const R1Desc *d, const uint32_t *tb, int nd, uint32_t tiles,
                           uint32_t grid, int round, int *err, cudaStream_t s);
cudaError_t launch_r1_scalar(int mode, const R1Desc *d, const uint32_t *tb, int nd, uint32_t grid, int round,
                             cudaStream_t s);

// Grover-mixer QAOA on cost degeneracies (kernels_grover.cu).
struct DegLaunch {
    uint64_t up_lo[128], up_hi[128];  // weight-k problems: all neighbours of u
    uint64_t adj[64];                 // MaxCut: all neighbours
    int deg[64];
    int n, k, m, kind, comp, n_bins;  // kind 0 MaxCut (2^n states), 1 DkS, 2 k-vertex cover
};
int grover_max_bins();
// Size of the enumerated set for the bit-sliced weight-k count (2..8), or 0
// when that kernel does not apply (MaxCut, degree-dependent costs, other sizes).
int degeneracy_sliced_kk(const DegLaunch &L);
// Counts the weight-KK sets {v} u T, v < min(T), for the (KK-1)-sets T of
// colex ranks [t_start, t_start + t_count).
cudaError_t launch_degeneracy_sliced(const DegLaunch &L, const uint64_t *d_binom, uint64_t t_start,
                                     uint64_t t_count, unsigned long long *d_counts, int *d_err, cudaStream_t s);
cudaError_t launch_degeneracy(const DegLaunch &L, const uint64_t *d_binom, uint64_t start, uint64_t count,
                              unsigned long long *d_counts, int *d_err, cudaStream_t s);
cudaError_t launch_grover_eval(const int64_t *d_counts, int nb, int p, int n_sets, const double *d_angles,
                               double *d_E, double *d_grad, cudaStream_t s);
int binom_table_max();
cudaError_t upload_binom_table();

}  // namespace qg
