// C ABI of the library (include/qaoa.h): context, scratch arena, argument
// validation, the pass schedule of the X mixer, launch planning and
// measurement hooks.  All arithmetic of the method runs in the kernels of
// kernels_xmix.cu / kernels_cost.cu / kernels_eig.cu; this file only decides
// what to launch on which buffers.
#include "qaoa.h"
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

using namespace qg;

namespace {

// NVTX range for the duration of a scope: entry points and kernel launches
// show up by name in a timeline tool; with no tool attached a push or pop is
// a pointer check.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct StatAcc {
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
    double flops = 0.0;
};

struct PendingEv {
    int fam;
    cudaEvent_t a, b;
};

// One unit of work: one angle set of one problem instance.
struct Unit {
    const void *cost;
    int cost_dtype;
    int n;
    int p;
    const double *angles;  // device, 2p
    double *E;             // device
    double *grad;          // device, 2p (gradient runs)
    const float2 *init;    // device or nullptr
    int tsize;             // phase-table entries (uint8 costs)
    int mixer_kind;        // QAOA_MIXER_X, _EIGEN, _EIGEN_SYM or _GROVER
    int job;               // job index (eigenbasis sets of one job form one GEMM group)
    int64_t dim;           // feasible-set size
    const float *V;        // eigenbasis mixer: D x D eigenvectors
    const double *lam;     // eigenbasis mixer: D eigenvalues
    int gemm_precision;
    int k;                 // block-diagonal XY mixer: Hamming weight of the feasible states
    uint64_t mixer_id;     // eigenbasis mixers: caller's id of (V, lambda); 0 = none
    int ma;                // X mixer with one angle per (round, qubit)
    int gm;                // general X mixer (Hadamard-basis weights wts)
    const double *wts;     // general X mixer: n + 1 weights
};

enum LaunchKind { LK_PREP, LK_SMALL, LK_XPASS, LK_REDUCE, LK_EIG_INIT, LK_EIG_GEMM, LK_COST_MEAN, LK_ORBIT,
                  LK_OPERANDS, LK_R1_PASS, LK_R1_SCALAR };

struct LaunchRec {
    int kind;
    int T = 0, bwd = 0, cost_dtype = 0, nbuf = 1, var = 0;
    size_t desc_off = 0, tb_off = 0;
    int ndesc = 0;
    uint32_t tiles = 0;
    int small_maxn = 0, small_grad = 0, t12 = 0;
    int fam = 0;
    double bytes = 0.0;
    double flops = 0.0;
    // eigenbasis mixer launches (parameters passed by value)
    EigEpiParams ep{};
    const float *gA = nullptr, *gB = nullptr;
    int Mp = 0, Np = 0, Kp = 0;
    float *iX = nullptr, *iX_lo = nullptr, *ick0 = nullptr;
    const float2 *iinit = nullptr;
    float iamp0 = 0.f;
    int tc = 0;        // tensor-core product (tensor maps below)
    CUtensorMap tm[4];  // A_hi, A_lo, B_hi, B_lo
    int sched_idx = -1;  // pass launches: tile counter slot
    int cost_free = 0;   // pass launches: no descriptor reads the cost
    int fused = 0;       // pass launches: round-boundary passes (PF_FUSED)
    double *mean_out = nullptr;  // LK_COST_MEAN: where the cost mean goes
    // Grover-mixer (rank-one) launches: mode, round and the pass grid, which
    // fixes the slot layout the following scalar launch reads
    int r1mode = 0, r1round = 0;
    uint32_t r1grid = 0;
    // grouped (block-diagonal) products and orbit kernels
    int grouped = 0, n_mtiles = 0, lda = 0, ldb = 0;
    const GroupTile *gtiles = nullptr;
    OrbitTabs otab{};
    OrbitArgs oarg{};
    // LK_OPERANDS: padded (and tf32-split) operand planes of an eigendecomposition
    struct {
        int sym;
        const float *V;
        const double *lam;
        int D, ld, nb, pmax;
        const int *bdim, *boff, *bpos;
        float *Vp, *Vtp, *Vpl, *Vtpl, *lam_hi, *lam_lo;
    } op{};
};

struct Plan {
    uint64_t key = 0;
    bool valid = false;
    std::vector<LaunchRec> launches;
    int n_sched = 0;  // pass launches (one tile counter each, zeroed per call)
    bool eig_tc = false;  // tensor-core eigenbasis products (split-K tail workspace)
};

// Global-bit layout of one pass: local bits 0..c-1 are global bits 0..c-1,
// local bits c..T-1 are global bits lo..lo+T-c-1.
struct Group {
    int c, lo;
};

constexpr int kMaxXQubits = 32;   // 32-bit element offsets in the pass kernel
constexpr int kMaxEigDim = 1 << 16; // feasible states of an eigenbasis mixer
constexpr int64_t kMaxGroverDim = 1ll << 36;  // feasible states of a Grover (rank-one) mixer
constexpr int kCminDefault = 4;   // >= 16 contiguous amplitudes = one 128-byte line
constexpr int kTmaSegBits = 8;    // shorter runs are fetched through a TMA tensor map
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Passes of one mixer round for n qubits and tile bits T: one contiguous pass
// over qubits 0..T-1, then the remaining n-T qubits in the fewest contiguous
// chunks of at most T-cmin qubits, each gathered with 2^c contiguous
// amplitudes (c = T - chunk >= cmin).  split: 0 = chunks as equal as
// possible, 1 = full chunks first and the remainder last, 2 = the remainder
// first.
std::vector<Group> make_groups(int n, int T, int cmin, int split) {
    std::vector<Group> g;
    g.push_back({T, T});
    const int R = n - T;
    if (R <= 0) return g;
    const int hmax = T - cmin;
    const int P = (R + hmax - 1) / hmax;
    const int rem = R - hmax * (P - 1);
    int lo = T;
    for (int j = 0; j < P; j++) {
        int h;
        if (split == 1) h = j < P - 1 ? hmax : rem;
        else if (split == 2) h = j == 0 ? rem : hmax;
        else h = R / P + (j < R % P ? 1 : 0);
        g.push_back({T - h, lo});
        lo += h;
    }
    return g;
}

// Minimum contiguous run (log2 amplitudes) of a gathered pass: 2^4 complex64
// amplitudes = one 128-byte line (and 16 bytes of uint8 cost, the bulk-copy
// granule).  QAOA_MIN_CONTIG overrides it for tuning sweeps (4..8).
int env_int(const char *name, int dflt, int lo, int hi) {
    const char *v = std::getenv(name);
    if (!v || !*v) return dflt;
    const int x = std::atoi(v);
    return (x < lo || x > hi) ? dflt : x;
}
// Round-boundary fusion of the X-mixer passes, as a mask of the boundary
// kinds fused: bit 0 boundaries on the contiguous group, bit 1 boundaries on
// a gathered group.  QAOA_FUSE selects 0 none, 1 all (default), 2 contiguous
// only, 3 gathered only, for comparison runs.
int fusion_mask() {
    static const int v = env_int("QAOA_FUSE", 1, 0, 3);
    static const int masks[4] = {0, 3, 1, 2};
    return masks[v];
}

// Tile buffers of the round-boundary adjoint passes (QAOA_FUSED_NBUF overrides
// it for tuning sweeps: 1 or 2).
int fused_bwd_nbuf() {
    static const int v = env_int("QAOA_FUSED_NBUF", 1, 1, 2);
    return v;
}

int min_contig() {
    static const int c = env_int("QAOA_MIN_CONTIG", kCminDefault, 4, 8);
    return c;
}

}  // namespace

struct qaoa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int *d_err = nullptr;
    std::map<std::string, Buf> bufs;
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    double *h_io = nullptr;
    size_t h_io_count = 0;
    bool profiling = false;
    std::vector<std::string> fam_names;
    std::map<std::string, int> fam_index;
    std::vector<StatAcc> fam_stats;
    std::vector<PendingEv> pending;
    std::vector<cudaEvent_t> ev_pool;
    int64_t launches = 0;
    Plan plan;
    std::set<std::string> eig_ready;  // prepared eigenbasis operands (by V, lambda, D)
    std::map<std::pair<int, int>, qaoa_xtune> xtune;  // X-mixer schedules by (n, cost dtype)
    uint64_t tune_epoch = 0;                          // bumped on every schedule change
    int ckpt_mode = QAOA_CKPT_PASS;                   // checkpointing of batched gradients
    int64_t state_limit = -1;                         // caller's cap on state scratch (-1: none)
    std::map<std::pair<int, int>, SymLayout> sym;     // cyclic-shift layouts by (n, k)
};

namespace {

bool valid_xtune(const qaoa_xtune &t) {
    return t.n > small_max_n() && t.n <= kMaxXQubits && (t.cost_dtype == QAOA_COST_F32 || t.cost_dtype == QAOA_COST_U8) &&
           t.cmin >= 4 && t.cmin <= 8 && t.split >= 0 && t.split <= 2 && (t.nbuf_bwd_contig == 1 || t.nbuf_bwd_contig == 2) &&
           (t.nbuf_bwd_gather == 1 || t.nbuf_bwd_gather == 2);
}

qaoa_status fail(qaoa_ctx *ctx, qaoa_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return st;
}

qaoa_status cuda_fail(qaoa_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, QAOA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QG_CUDA(ctx, call, what)                          \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, what); \
    } while (0)

int family(qaoa_ctx *ctx, const std::string &name) {
    auto it = ctx->fam_index.find(name);
    if (it != ctx->fam_index.end()) return it->second;
    const int id = (int)ctx->fam_names.size();
    ctx->fam_names.push_back(name);
    ctx->fam_stats.push_back(StatAcc());
    ctx->fam_index[name] = id;
    return id;
}

cudaEvent_t take_event(qaoa_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool capturing(qaoa_ctx *ctx) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cs);
    return cs != cudaStreamCaptureStatusNone;
}

// Split-K tail of the tensor-core eigenbasis products: counters, then the
// partial tiles (see launch_eig_gemm_tc).
size_t eig_split_cnt_bytes() { return ((size_t)eig_split_max_tail() * sizeof(unsigned) + 255) / 256 * 256; }
size_t eig_split_bytes() {
    return eig_split_cnt_bytes() + (size_t)eig_split_max_tail() * kEigMaxSeg * kEigTile * kEigTile * sizeof(float);
}

// Device scratch by name; grows (never shrinks) and invalidates the cached
// plan when a buffer moves.
qaoa_status scratch(qaoa_ctx *ctx, const char *name, size_t bytes, void **out) {
    Buf &b = ctx->bufs[name];
    if (b.bytes >= bytes && b.p) {
        *out = b.p;
        return QAOA_OK;
    }
    if (capturing(ctx))
        return fail(ctx, QAOA_ERR_INVALID,
                    "scratch '%s' must grow during stream capture; run the call once uncaptured first",
                    name);
    if (b.p) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    ctx->plan.valid = false;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, kAlign));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, QAOA_ERR_OOM, "cannot allocate %.3f GiB of scratch for '%s'",
                    bytes / 1073741824.0, name);
    }
    b.p = p;
    b.bytes = std::max<size_t>(bytes, kAlign);
    *out = p;
    return QAOA_OK;
}

qaoa_status host_stage(qaoa_ctx *ctx, size_t bytes) {
    if (ctx->h_stage_bytes >= bytes) return QAOA_OK;
    if (ctx->h_stage) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeHost(ctx->h_stage);
    }
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    QG_CUDA(ctx, cudaMallocHost(&ctx->h_stage, bytes), "cudaMallocHost");
    ctx->h_stage_bytes = bytes;
    return QAOA_OK;
}

// --------------------------------------------------------- tensor maps
// cuTensorMapEncodeTiled from the driver through the runtime (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Gathered tile of a 2^n-element vector: 2^c contiguous elements (dim 0),
// the free bits c..lo-1 (dim 1), the 2^(T-c) rows of the gathered qubits
// lo..lo+T-c-1 (dim 2), the free bits above them (dim 3).
bool encode_gather_map(CUtensorMap *m, const void *base, int n, int c, int lo, int elsz) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const int h = kPassTileBits - c;
    const cuuint64_t dims[4] = {1ull << c, 1ull << (lo - c), 1ull << h, 1ull << (n - lo - h)};
    const cuuint64_t strides[3] = {(1ull << c) * elsz, (1ull << lo) * elsz, (1ull << (lo + h)) * elsz};
    const cuuint32_t box[4] = {1u << c, 1u, 1u << h, 1u};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = elsz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : elsz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                               : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    return enc(m, dt, 4, const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row-major float32 matrix [rows][ld] as a K-major tensor-core operand:
// 32-float (128-byte) boxes x 128 rows, 128-byte swizzle.
bool encode_kmajor_map(CUtensorMap *m, const float *base, int ld, int rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {32, 128};
    const cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------- planning

struct UnitLayout {
    int T_f, T_b;
    std::vector<Group> gf, gb;
    uint32_t tiles_f, tiles_b;
    int64_t stride;  // partial slots per quantity
    int ckpt;        // QAOA_CKPT_* actually used
    int vecs;        // state vectors held in scratch
    int nb_bc, nb_bg;  // adjoint tile buffers (contiguous / gathered passes)
    bool fused;      // alternating group order, some round boundaries fused (fuse_mask)
    int fuse_mask;   // boundary kinds fused: bit 0 contiguous group, bit 1 gathered
};

// Whether the boundary between rounds k and k+1 is one fused pass.  With the
// alternating order round k ends on group P-1 (k even) or group 0 (k odd).
bool boundary_fused(const UnitLayout &L, int k) {
    if (!L.fused) return false;
    const int g = (k & 1) ? 0 : (int)L.gf.size() - 1;
    return (L.fuse_mask & (L.gf[g].c >= kPassTileBits ? 1 : 2)) != 0;
}

qaoa_xtune default_xtune(int n, int dt) {
    qaoa_xtune t;
    std::memset(&t, 0, sizeof(t));
    t.n = n;
    t.cost_dtype = dt;
    t.cmin = min_contig();
    t.split = 0;
    t.nbuf_bwd_contig = 1;
    t.nbuf_bwd_gather = 1;
    return t;
}

qaoa_xtune tune_for(const qaoa_ctx *ctx, int n, int dt) {
    auto it = ctx->xtune.find({n, dt});
    return it != ctx->xtune.end() ? it->second : default_xtune(n, dt);
}

// Forward passes of a unit: P per round, one fewer per fused round boundary.
int forward_passes(const UnitLayout &L, int p) {
    int n = p * (int)L.gf.size();
    for (int k = 0; k + 1 < p; k++) n -= boundary_fused(L, k) ? 1 : 0;
    return n;
}

int layout_vecs(const UnitLayout &L, int p, bool grad) {
    if (!grad) return 1;
    if (L.ckpt == QAOA_CKPT_PASS) return 1 + forward_passes(L, p);
    if (L.ckpt == QAOA_CKPT_ROUND) return 2 + (p - 1);
    return 2;
}

UnitLayout layout_for(const qaoa_ctx *ctx, const Unit &u, bool grad, int ckpt) {
    const qaoa_xtune t = tune_for(ctx, u.n, u.cost_dtype);
    UnitLayout L;
    L.T_f = kPassTileBits;
    L.T_b = kPassTileBits;
    L.gf = make_groups(u.n, L.T_f, t.cmin, t.split);
    if (u.gm) {  // general X mixer: two half rounds of the same passes
        const std::vector<Group> h = L.gf;
        L.gf.insert(L.gf.end(), h.begin(), h.end());
    }
    L.gb = L.gf;  // per-pass checkpoints pair forward and adjoint passes one to one
    L.tiles_f = 1u << (u.n - L.T_f);
    L.tiles_b = 1u << (u.n - L.T_b);
    L.stride = std::max<int64_t>(L.tiles_f, (int64_t)L.gb.size() * (u.ma ? kPassTileBits : 1) * L.tiles_b) *
               kPassWarps;
    L.ckpt = grad ? (u.gm ? QAOA_CKPT_PASS : ckpt) : QAOA_CKPT_NONE;  // general mixer: per-pass only
    // fused round boundaries: transverse field, per-pass checkpoints (or no gradient)
    L.fuse_mask = fusion_mask();
    L.fused = L.fuse_mask != 0 && !u.ma && !u.gm && L.gf.size() >= 2 && u.p >= 2 &&
              (!grad || L.ckpt == QAOA_CKPT_PASS);
    L.vecs = layout_vecs(L, u.p, grad);
    L.nb_bc = t.nbuf_bwd_contig;
    L.nb_bg = t.nbuf_bwd_gather;
    return L;
}

void fill_geometry(PassDesc &d, int n, int T, const Group &g) {
    d.n = (uint8_t)n;
    bool used[64] = {false};
    for (int j = 0; j < T; j++) {
        const int gp = j < g.c ? j : g.lo + (j - g.c);
        d.gpos[j] = (uint8_t)gp;
        used[gp] = true;
    }
    int nf = 0;
    for (int b = 0; b < n; b++)
        if (!used[b]) d.fpos[nf++] = (uint8_t)b;
    d.nfree = (uint8_t)nf;
    d.c = (uint8_t)g.c;
    d.ntiles = 1u << nf;
    d.active = (g.c == T) ? ((1u << T) - 1u) : (((1u << T) - 1u) & ~((1u << g.c) - 1u));
}

double pass_bytes(const PassDesc &d, int bwd, int cost_bytes) {
    const double N = std::ldexp(1.0, d.n);
    double b = 0.0;
    if (!bwd) {
        if (!(d.flags & PF_GEN_INIT)) b += 8;
        if (d.psi_out) b += 8;
        if (d.flags & (PF_PHASE | PF_FUSED)) b += cost_bytes;
        if (d.flags & PF_E) b += cost_bytes;
    } else {
        b += 8;  // psi
        if (!(d.flags & PF_LAM_FROM_C)) b += 8;
        else b += cost_bytes;
        if (d.flags & (PF_PHASE | PF_FUSED)) b += cost_bytes;
        if (d.psi_out) b += 8;
        if (d.lam_out) b += 8;
    }
    return b * N;
}

// Descriptors of every pass of one unit: forward rounds, then adjoint rounds
// in reverse.  Buffers: W = running state, L = adjoint state, CK[k] = state
// after round k (0-based, k < p-1) with per-round checkpoints; with per-pass
// checkpoints CK[k Pf + g] = output of forward pass g of round k (W unused).
void unit_passes(const Unit &u, const UnitLayout &L, bool grad, float2 *W, float2 *Lam, float2 *CK,
                 const RoundCoef *coef, const float2 *table, const float4 *wtab, double *part,
                 std::vector<PassDesc> &fwd, std::vector<PassDesc> &bwd) {
    const int p = u.p;
    const int64_t N = 1ll << u.n;
    const int Pf = (int)L.gf.size(), Pb = (int)L.gb.size();
    const float amp0 = (float)(1.0 / std::sqrt(std::ldexp(1.0, u.n)));
    const int ckpt = L.ckpt;
    const int nbq = u.ma ? u.n : 1;                               // coefficients per round
    const int64_t bslot = (u.ma ? kPassTileBits : 1) * (int64_t)L.tiles_b * kPassWarps;  // beta partials per pass
    auto ck = [&](int k) { return CK + (int64_t)k * N; };
    auto pk = [&](int k, int g) { return CK + ((int64_t)k * Pf + g) * N; };
    if (u.gm) {
        // general X mixer: passes j = 0..2P-1 of round k are the half rounds
        // e^{-i (pi/4) X} (j < P, coefficient 2k, phase on the first) and
        // e^{+i (pi/4) X} (j >= P, coefficient 2k + 1), the weight phases
        // e^{-i b_k G} on the load of pass P
        const int P = Pf / 2;
        const int64_t nw = u.n + 1;
        auto fwd_desc = [&](int k, int j) {
            PassDesc d;
            std::memset(&d, 0, sizeof(d));
            fill_geometry(d, u.n, L.T_f, L.gf[j]);
            d.cost = u.cost;
            d.coef = coef + 2 * k + (j >= P ? 1 : 0);
            d.table = table ? table + (int64_t)k * kPhaseTable : nullptr;
            d.wtab = wtab + (int64_t)k * nw;
            d.amp0 = amp0;
            if (j == 0) d.flags |= PF_PHASE;
            if (j == P) d.flags |= PF_WDIAG;
            return d;
        };
        for (int k = 0; k < p; k++) {
            for (int j = 0; j < Pf; j++) {
                PassDesc d = fwd_desc(k, j);
                const bool first = k == 0 && j == 0, last = k == p - 1 && j == Pf - 1;
                if (first) {
                    if (u.init) {
                        d.psi_in = u.init;
                        d.flags |= PF_TWIST_IN;
                    } else {
                        d.flags |= PF_GEN_INIT;
                    }
                } else {
                    d.psi_in = grad ? (j == 0 ? pk(k - 1, Pf - 1) : pk(k, j - 1)) : W;
                }
                if (last) {
                    d.flags |= PF_E;
                    d.part_E = part;
                }
                d.psi_out = grad ? pk(k, j) : (last ? nullptr : W);
                fwd.push_back(d);
            }
        }
        if (!grad) return;
        for (int k = p - 1; k >= 0; k--) {
            for (int j = Pf - 1; j >= 0; j--) {
                PassDesc d = fwd_desc(k, j);
                d.flags &= PF_PHASE | PF_WDIAG;
                d.psi_in = pk(k, j);
                if (k == p - 1 && j == Pf - 1) d.flags |= PF_LAM_FROM_C;
                else d.lam_in = Lam;
                d.lam_out = (k == 0 && j == 0) ? nullptr : Lam;
                if (j == P) d.part_beta = part + (int64_t)(1 + k) * L.stride;
                if (j == 0) d.part_gamma = part + (int64_t)(1 + p + k) * L.stride;
                bwd.push_back(d);
            }
        }
        return;
    }
    if (L.fused) {
        // Alternating group order: even rounds run groups 0 .. P-1, odd rounds
        // P-1 .. 0, so round k ends on the group round k+1 starts with and the
        // two meet in one round-boundary pass (PF_FUSED), which also applies
        // round k+1's phase.  Forward pass j writes checkpoint j (gradients)
        // or works in place on W (expectation only).
        struct FP {
            int g, k, fused;  // group, round (fused: rounds k and k+1)
            int first;        // the first pass of round k (not fused): applies / undoes its phase
        };
        std::vector<FP> seq;
        auto group_at = [&](int k, int q) { return (k & 1) ? Pf - 1 - q : q; };  // q-th group of round k
        for (int k = 0; k < p; k++) {
            const int q0 = (k > 0 && boundary_fused(L, k - 1)) ? 1 : 0;
            for (int q = q0; q < Pf; q++)
                seq.push_back({group_at(k, q), k, (q == Pf - 1 && k < p - 1 && boundary_fused(L, k)) ? 1 : 0,
                               q == 0 ? 1 : 0});
        }
        const int J = (int)seq.size();
        auto pj = [&](int j) { return CK + (int64_t)j * N; };
        auto slot = [&](int k, int g) {  // round k's beta partial slot of group g
            const int q = (k & 1) ? Pf - 1 - g : g;
            return part + (int64_t)(1 + k) * L.stride + (int64_t)q * bslot;
        };
        auto base_desc = [&](const FP &f) {
            PassDesc d;
            std::memset(&d, 0, sizeof(d));
            fill_geometry(d, u.n, L.T_f, L.gf[f.g]);
            d.cost = u.cost;
            d.coef = coef + (int64_t)f.k * nbq;
            const int tk = f.fused ? f.k + 1 : f.k;  // the round whose phase the pass applies
            d.table = table ? table + (int64_t)tk * kPhaseTable : nullptr;
            d.amp0 = amp0;
            if (f.fused) {
                d.flags |= PF_FUSED;
                d.coef2 = coef + (int64_t)(f.k + 1) * nbq;
            }
            return d;
        };
        for (int j = 0; j < J; j++) {
            PassDesc d = base_desc(seq[j]);
            if (seq[j].first) d.flags |= PF_PHASE;
            if (j == 0) {
                if (u.init) {
                    d.psi_in = u.init;
                    d.flags |= PF_TWIST_IN;
                } else {
                    d.flags |= PF_GEN_INIT;
                }
            } else {
                d.psi_in = grad ? pj(j - 1) : W;
            }
            if (j == J - 1) {
                d.flags |= PF_E;
                d.part_E = part;
            }
            d.psi_out = grad ? pj(j) : (j == J - 1 ? nullptr : W);
            fwd.push_back(d);
        }
        if (!grad) return;
        for (int j = J - 1; j >= 0; j--) {
            const FP &f = seq[j];
            PassDesc d = base_desc(f);
            d.psi_in = pj(j);
            if (j == J - 1) d.flags |= PF_LAM_FROM_C;
            else d.lam_in = Lam;
            d.lam_out = j > 0 ? Lam : nullptr;
            if (f.fused) {
                d.part_beta = slot(f.k + 1, f.g);
                d.part_beta2 = slot(f.k, f.g);
                d.part_gamma = part + (int64_t)(1 + p + f.k + 1) * L.stride;
            } else {
                d.part_beta = slot(f.k, f.g);
            }
            if (f.first) {
                d.flags |= PF_PHASE;
                d.part_gamma = part + (int64_t)(1 + p + f.k) * L.stride;
            }
            bwd.push_back(d);
        }
        return;
    }
    if (grad && ckpt == QAOA_CKPT_PASS) {
        for (int k = 0; k < p; k++) {
            for (int g = 0; g < Pf; g++) {
                PassDesc d;
                std::memset(&d, 0, sizeof(d));
                fill_geometry(d, u.n, L.T_f, L.gf[g]);
                d.cost = u.cost;
                d.coef = coef + (int64_t)k * nbq;
                d.table = table ? table + (int64_t)k * kPhaseTable : nullptr;
                d.amp0 = amp0;
                if (g == 0) {
                    d.flags |= PF_PHASE;
                    if (k == 0) {
                        if (u.init) {
                            d.psi_in = u.init;
                            d.flags |= PF_TWIST_IN;
                        } else {
                            d.flags |= PF_GEN_INIT;
                        }
                    } else {
                        d.psi_in = pk(k - 1, Pf - 1);
                    }
                } else {
                    d.psi_in = pk(k, g - 1);
                }
                if (g == Pf - 1 && k == p - 1) {
                    d.flags |= PF_E;
                    d.part_E = part;
                }
                d.psi_out = pk(k, g);
                fwd.push_back(d);
            }
        }
        // adjoint: pass (k, g) reads the forward output of pass (k, g) and
        // writes lambda only; the next one reads the forward output before it
        for (int k = p - 1; k >= 0; k--) {
            for (int q = 0; q < Pb; q++) {
                const int g = Pb - 1 - q;
                PassDesc d;
                std::memset(&d, 0, sizeof(d));
                fill_geometry(d, u.n, L.T_b, L.gb[g]);
                d.cost = u.cost;
                d.coef = coef + (int64_t)k * nbq;
                d.table = table ? table + (int64_t)k * kPhaseTable : nullptr;
                d.amp0 = amp0;
                d.psi_in = pk(k, g);
                if (k == p - 1 && q == 0) d.flags |= PF_LAM_FROM_C;
                else d.lam_in = Lam;
                if (g == 0) {
                    d.flags |= PF_PHASE;
                    d.part_gamma = part + (int64_t)(1 + p + k) * L.stride;
                    d.lam_out = k > 0 ? Lam : nullptr;
                } else {
                    d.lam_out = Lam;
                }
                d.part_beta = part + (int64_t)(1 + k) * L.stride + (int64_t)q * bslot;
                bwd.push_back(d);
            }
        }
        return;
    }
    for (int k = 0; k < p; k++) {
        for (int g = 0; g < Pf; g++) {
            PassDesc d;
            std::memset(&d, 0, sizeof(d));
            fill_geometry(d, u.n, L.T_f, L.gf[g]);
            d.cost = u.cost;
            d.coef = coef + (int64_t)k * nbq;
            d.table = table ? table + (int64_t)k * kPhaseTable : nullptr;
            d.amp0 = amp0;
            const bool first = g == 0, last = g == Pf - 1;
            if (first) {
                d.flags |= PF_PHASE;
                if (k == 0) {
                    if (u.init) {
                        d.psi_in = u.init;
                        d.flags |= PF_TWIST_IN;
                    } else {
                        d.flags |= PF_GEN_INIT;
                    }
                } else {
                    d.psi_in = (grad && ckpt) ? ck(k - 1) : W;
                }
            } else {
                d.psi_in = W;
            }
            if (last && k == p - 1) {
                d.flags |= PF_E;
                d.part_E = part;
                d.psi_out = grad ? W : nullptr;
            } else if (last && grad && ckpt) {
                d.psi_out = ck(k);
            } else {
                d.psi_out = W;
            }
            fwd.push_back(d);
        }
    }
    if (!grad) return;
    // Adjoint rounds in reverse.  Within a round the groups run in reverse
    // order, so the phase (gamma partial, undone phase) rides on the
    // contiguous group 0, the last pass of the round.
    for (int k = p - 1; k >= 0; k--) {
        for (int q = 0; q < Pb; q++) {
            const int g = Pb - 1 - q;
            PassDesc d;
            std::memset(&d, 0, sizeof(d));
            fill_geometry(d, u.n, L.T_b, L.gb[g]);
            d.cost = u.cost;
            d.coef = coef + (int64_t)k * nbq;
            d.table = table ? table + (int64_t)k * kPhaseTable : nullptr;
            d.amp0 = amp0;
            const bool first_round = k == p - 1;
            const bool last = q == Pb - 1;
            if (q == 0) {
                d.psi_in = (first_round || !ckpt) ? W : ck(k);
                if (first_round) d.flags |= PF_LAM_FROM_C;
                else d.lam_in = Lam;
            } else {
                d.psi_in = W;
                d.lam_in = Lam;
            }
            if (last) {
                d.flags |= PF_PHASE;
                d.part_gamma = part + (int64_t)(1 + p + k) * L.stride;
                if (!ckpt && k > 0) {
                    d.flags |= PF_UNPHASE_PSI;
                    d.psi_out = W;
                }
                d.lam_out = k > 0 ? Lam : nullptr;
            } else {
                d.psi_out = W;
                d.lam_out = Lam;
            }
            d.part_beta = part + (int64_t)(1 + k) * L.stride + (int64_t)q * bslot;
            bwd.push_back(d);
        }
    }
}

cudaError_t enqueue_operands(const LaunchRec &r, cudaStream_t s) {
    if (r.op.sym)
        return launch_sym_prepare(r.op.V, r.op.lam, r.op.bdim, r.op.boff, r.op.bpos, r.op.nb, r.op.pmax, r.op.Vp,
                                  r.op.Vtp, r.op.Vpl, r.op.Vtpl, r.op.lam_hi, r.op.lam_lo, s);
    return launch_eig_prepare(r.op.V, r.op.D, r.op.ld, r.op.Vp, r.op.Vtp, r.op.Vpl, r.op.Vtpl, r.op.lam, r.op.lam_hi,
                              r.op.lam_lo, s);
}

// Operand planes of a mixer with an id, built once when the plan is made.
qaoa_status launch_operands(qaoa_ctx *ctx, const LaunchRec &r) {
    cudaError_t e = enqueue_operands(r, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "eigenbasis preparation");
    QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "eigenbasis preparation");
    ctx->launches++;
    return QAOA_OK;
}

// Launches of one job of a block-diagonal XY mixer (QAOA_MIXER_EIGEN_SYM):
// the S angle sets are the columns of every product, all state matrices are in
// the momentum basis of the cyclic shift ([2 Spad][ldp], Re and Im rows), and
// the orbit kernel moves to and from the computational basis at each round
// boundary.  Per forward round r:
//   Y = e^{-i b_r lambda} (V_b^T X)   (grouped product; checkpoint V_b^T X)
//   Z = V_b Y                         (grouped product, plain store; with
//                                      gradients straight into checkpoint P_{r+1})
//   X = T^T e^{-i g_{r+1} C} T Z      (orbit kernel; last round: <C>, L)
// and per adjoint round r = p-1 .. 0:
//   Y = e^{+i b_r lambda} (V_b^T L)   (beta partials)
//   W = V_b Y
//   L = T^T e^{+i g_r C} T W          (gamma partials with P_r)
template <typename AddRed>
qaoa_status plan_sym_job(qaoa_ctx *ctx, const std::vector<Unit> &units, int u0, int S, int Spad, bool grad,
                         const SymLayout &SL, int nmt, int nob, char *st_base, double *part, double *c0,
                         const RoundCoef *coef, std::vector<LaunchRec> &Lr, AddRed &add_reduction, bool &any_tc) {
    const Unit &u = units[u0];
    const int p = u.p, ldp = SL.ldp, pmax = SL.pmax, NB = (int)SL.block_dim.size();
    const bool tcp = u.gemm_precision == QAOA_GEMM_3XTF32;
    // ---- device tables of the layout (uploaded once per context)
    char nm[128];
    snprintf(nm, sizeof(nm), "symtab:%d:%d", SL.n, SL.k);
    const std::string tkey = nm;
    std::vector<int> ints;
    auto put_ints = [&](const std::vector<int> &v) {
        const size_t off = ints.size();
        ints.insert(ints.end(), v.begin(), v.end());
        while (ints.size() % 4) ints.push_back(0);
        return off;
    };
    const size_t o_start = put_ints(SL.orb_start), o_mem = put_ints(SL.members), o_pos = put_ints(SL.vec_pos),
                 o_mroff = put_ints(SL.mr_off), o_bdim = put_ints(SL.block_dim), o_boff = put_ints(SL.block_off),
                 o_bpos = put_ints(SL.block_pos);
    std::vector<GroupTile> tiles;
    for (int b = 0; b < NB; b++) {
        const int P = SL.block_pos[b + 1] - SL.block_pos[b];
        for (int mt = 0; mt < P / kEigTile; mt++) {
            GroupTile t;
            t.a_row = SL.block_pos[b] + mt * kEigTile;
            t.k_off = SL.block_pos[b];
            t.kext = P;
            t.out_row = t.a_row;
            t.row_end = SL.block_pos[b] + SL.block_dim[b];
            t.part_idx = t.a_row / kEigTile;
            tiles.push_back(t);
        }
    }
    // longest K first, so the short blocks fill the last wave
    std::stable_sort(tiles.begin(), tiles.end(), [](const GroupTile &a, const GroupTile &b) { return a.kext > b.kext; });
    const size_t ints_b = align_up(ints.size() * sizeof(int)), mr_b = align_up(SL.mr.size() * sizeof(float)),
                 tiles_b = align_up(tiles.size() * sizeof(GroupTile));
    void *d_tab = nullptr;
    qaoa_status st = scratch(ctx, tkey.c_str(), ints_b + mr_b + tiles_b, &d_tab);
    if (st) return st;
    char *tb = static_cast<char *>(d_tab);
    const int *di = reinterpret_cast<const int *>(tb);
    const float *dmr = reinterpret_cast<const float *>(tb + ints_b);
    const GroupTile *dtiles = reinterpret_cast<const GroupTile *>(tb + ints_b + mr_b);
    if (!ctx->eig_ready.count(tkey)) {
        std::vector<char> img(ints_b + mr_b + tiles_b, 0);
        std::memcpy(img.data(), ints.data(), ints.size() * sizeof(int));
        for (size_t i = 0; i < SL.mr.size(); i++) reinterpret_cast<float *>(img.data() + ints_b)[i] = (float)SL.mr[i];
        std::memcpy(img.data() + ints_b + mr_b, tiles.data(), tiles.size() * sizeof(GroupTile));
        QG_CUDA(ctx, cudaMemcpy(d_tab, img.data(), img.size(), cudaMemcpyHostToDevice), "layout upload");
        ctx->eig_ready.insert(tkey);
    }
    OrbitTabs T;
    T.orb_start = di + o_start;
    T.members = di + o_mem;
    T.vec_pos = di + o_pos;
    T.mr = dmr;
    T.mr_off = di + o_mroff;
    T.n_orbits = SL.n_orbits;
    T.max_r = SL.n;
    T.mr_len = (int)SL.mr.size();
    if (T.mr_len > kOrbitSmem)
        return fail(ctx, QAOA_ERR_UNSUPPORTED, "orbit matrices of n=%d exceed the kernel's shared memory", SL.n);
    // ---- operand planes of (V_b, lambda), prepared once per (V, lambda, n, k)
    // (kept across calls for a mixer with an id, else rebuilt by every call)
    if (u.mixer_id)
        snprintf(nm, sizeof(nm), "symV:id%llu:%d:%d:%d", (unsigned long long)u.mixer_id, SL.n, SL.k, tcp ? 1 : 0);
    else
        snprintf(nm, sizeof(nm), "symV:call:%d:%d:%d", SL.n, SL.k, tcp ? 1 : 0);
    const std::string key = nm;
    const size_t plane = (size_t)ldp * pmax * sizeof(float);
    void *dV = nullptr, *dVt = nullptr, *dVl = nullptr, *dVtl = nullptr, *dL = nullptr;
    if ((st = scratch(ctx, (key + ":V").c_str(), plane, &dV)) || (st = scratch(ctx, (key + ":Vt").c_str(), plane, &dVt)))
        return st;
    if (tcp && ((st = scratch(ctx, (key + ":Vlo").c_str(), plane, &dVl)) ||
                (st = scratch(ctx, (key + ":Vtlo").c_str(), plane, &dVtl))))
        return st;
    if ((st = scratch(ctx, (key + ":lam").c_str(), (size_t)2 * ldp * sizeof(float), &dL))) return st;
    float *lam_hi = static_cast<float *>(dL), *lam_lo = lam_hi + ldp;
    if (!u.mixer_id || !ctx->eig_ready.count(key)) {
        LaunchRec r;
        r.kind = LK_OPERANDS;
        r.op.sym = 1;
        r.op.V = u.V;
        r.op.lam = u.lam;
        r.op.nb = NB;
        r.op.pmax = pmax;
        r.op.bdim = di + o_bdim;
        r.op.boff = di + o_boff;
        r.op.bpos = di + o_bpos;
        r.op.Vp = static_cast<float *>(dV);
        r.op.Vtp = static_cast<float *>(dVt);
        r.op.Vpl = static_cast<float *>(dVl);
        r.op.Vtpl = static_cast<float *>(dVtl);
        r.op.lam_hi = lam_hi;
        r.op.lam_lo = lam_lo;
        r.fam = family(ctx, "eig_operands");
        if (u.mixer_id) {
            st = launch_operands(ctx, r);
            if (st) return st;
            ctx->eig_ready.insert(key);
        } else {
            Lr.push_back(r);
        }
    }
    const float *Vp = static_cast<const float *>(dV), *Vtp = static_cast<const float *>(dVt);
    const float *Vpl = static_cast<const float *>(dVl), *Vtpl = static_cast<const float *>(dVtl);
    // ---- state matrices: X, Y, L, Z, 2p checkpoints (CKY: V_b^T X of each
    // round, P: the state entering each round), remainder planes last
    const size_t mat = (size_t)2 * Spad * ldp;
    float *base = reinterpret_cast<float *>(st_base);
    float *X = base, *Y = base + mat, *Lm = grad ? base + 2 * mat : nullptr;
    float *Z = base + (grad ? 3 : 2) * mat;
    auto CKY = [&](int r) { return base + (4 + r) * mat; };
    auto CKP = [&](int r) { return base + (4 + p + r) * mat; };
    const int lo0 = grad ? 4 + 2 * p : 3;
    float *Xl = tcp ? base + lo0 * mat : nullptr;
    float *Yl = tcp ? base + (lo0 + 1) * mat : nullptr;
    float *Ll = (tcp && grad) ? base + (lo0 + 2) * mat : nullptr;
    const int nmat = (grad ? 3 + 2 * p + 3 * (tcp ? 1 : 0) : 2 + 2 * (tcp ? 1 : 0)) + 1;
    // padding entries are never written: clear the matrices once per plan
    QG_CUDA(ctx, cudaMemsetAsync(base, 0, mat * nmat * sizeof(float), ctx->stream), "state clear");
    const int64_t pq = (int64_t)Spad * std::max(nmt, nob);  // partial slots per quantity
    EigEpiParams ep{};
    ep.M = SL.D;
    ep.ld = ldp;
    ep.nsets = S;
    ep.lam_hi = lam_hi;
    ep.lam_lo = lam_lo;
    ep.cost = u.cost;
    ep.cost_dtype = u.cost_dtype;
    ep.coef = coef;
    ep.coef_stride = p;
    ep.part_stride = nmt;
    double useful = 0.0;  // useful flops of one grouped product
    for (int b = 0; b < NB; b++) useful += 2.0 * SL.block_dim[b] * (double)SL.block_dim[b] * 2.0 * S;
    const int fam_g = family(ctx, tcp ? "eig_gemm_tc_3xtf32_blocks" : "eig_gemm_simt_blocks");
    const int fam_o = family(ctx, "orbit_transform");
    bool map_ok = true;
    auto lo_of = [&](const float *B) -> const float * { return B == X ? Xl : B == Y ? Yl : B == Lm ? Ll : nullptr; };
    auto gemm = [&](const float *A, const float *B, EigEpiParams q) {
        LaunchRec r;
        r.kind = LK_EIG_GEMM;
        r.grouped = 1;
        r.gtiles = dtiles;
        r.n_mtiles = (int)tiles.size();
        r.gA = A;
        r.gB = B;
        r.lda = pmax;
        r.ldb = ldp;
        r.Np = 2 * Spad;
        r.flops = useful;
        r.fam = fam_g;
        if (tcp) {
            r.tc = 1;
            any_tc = true;
            const float *Al = A == Vp ? Vpl : Vtpl;
            map_ok = map_ok && encode_kmajor_map(&r.tm[0], A, pmax, ldp) && encode_kmajor_map(&r.tm[1], Al, pmax, ldp) &&
                     encode_kmajor_map(&r.tm[2], B, ldp, 2 * Spad) &&
                     encode_kmajor_map(&r.tm[3], lo_of(B), ldp, 2 * Spad);
            q.out_lo = q.out == Y ? Yl : nullptr;  // only Y feeds another product
        }
        r.ep = q;
        Lr.push_back(r);
    };
    auto orbit = [&](const OrbitArgs &a) {
        LaunchRec r;
        r.kind = LK_ORBIT;
        r.otab = T;
        r.oarg = a;
        r.fam = fam_o;
        // algorithmic bytes: the matrices read and written once
        r.bytes = 4.0 * 2 * S * SL.D * ((a.in ? 1 : 0) + (a.in_psi ? 1 : 0) + (a.out ? (a.out_lo ? 2 : 1) : 0) +
                                        (a.ckpt ? 1 : 0));
        Lr.push_back(r);
    };
    OrbitArgs oa{};
    oa.D = SL.D;
    oa.ldp = ldp;
    oa.nsets = S;
    oa.amp0 = (float)(1.0 / std::sqrt((double)SL.D));
    oa.cost = u.cost;
    oa.cost_dtype = u.cost_dtype;
    oa.coef = coef;
    oa.coef_stride = p;
    oa.part_stride = nob;
    if (grad) {
        LaunchRec r;
        r.kind = LK_COST_MEAN;
        r.ep = ep;
        r.mean_out = c0;
        r.fam = family(ctx, "cost_mean");
        Lr.push_back(r);
    }
    {
        OrbitArgs a = oa;
        a.mode = ORB_INIT;
        a.round = 0;
        a.out = X;
        a.out_lo = Xl;
        a.ckpt = grad ? CKP(0) : nullptr;
        a.init = u.init;
        orbit(a);
    }
    for (int r = 0; r < p; r++) {
        EigEpiParams q = ep;
        q.kind = EPI_FWD_EIG;
        q.round = r;
        q.out = Y;
        q.ckpt = grad ? CKY(r) : nullptr;
        gemm(Vtp, X, q);
        float *zout = (grad && r < p - 1) ? CKP(r + 1) : Z;
        q = ep;
        q.kind = EPI_STORE;
        q.out = zout;
        gemm(Vp, Y, q);
        OrbitArgs a = oa;
        a.in = zout;
        if (r < p - 1) {
            a.mode = ORB_PHASE;
            a.round = r + 1;
            a.out = X;
            a.out_lo = Xl;
        } else {
            a.mode = ORB_LAST;
            a.round = r;
            a.out = grad ? Lm : nullptr;
            a.out_lo = grad ? Ll : nullptr;
            a.c0 = grad ? c0 : nullptr;
            a.part = part;
        }
        orbit(a);
    }
    if (grad) {
        for (int r = p - 1; r >= 0; r--) {
            EigEpiParams q = ep;
            q.kind = EPI_BWD_EIG;
            q.round = r;
            q.out = Y;
            q.ck_in = CKY(r);
            q.part = part + (1 + r) * pq;
            gemm(Vtp, Lm, q);
            q = ep;
            q.kind = EPI_STORE;
            q.out = Z;
            gemm(Vp, Y, q);
            OrbitArgs a = oa;
            a.mode = ORB_BWD;
            a.round = r;
            a.in = Z;
            a.in_psi = CKP(r);
            a.out = r > 0 ? Lm : nullptr;
            a.out_lo = r > 0 ? Ll : nullptr;
            a.c0 = c0;
            a.part = part + (1 + p + r) * pq;
            orbit(a);
        }
    }
    if (!map_ok) return fail(ctx, QAOA_ERR_CUDA, "tensor map encoding failed");
    for (int s2 = 0; s2 < S; s2++) {
        const Unit &us = units[u0 + s2];
        add_reduction(part + (int64_t)s2 * nob, nob, us.E, 1.0);
        if (grad)
            for (int r = 0; r < p; r++) {
                add_reduction(part + (1 + r) * pq + (int64_t)s2 * nmt, nmt, us.grad + r, 2.0);
                add_reduction(part + (1 + p + r) * pq + (int64_t)s2 * nob, nob, us.grad + p + r, 2.0);
            }
    }
    return QAOA_OK;
}

const char *dtype_name(int dt) { return dt == QAOA_COST_U8 ? "u8" : "f32"; }

// Build (or reuse) the launch plan for a unit list and enqueue it.
qaoa_status run_units(qaoa_ctx *ctx, const std::vector<Unit> &units, bool grad, int ckpt) {
    uint64_t key = fnv1a(units.data(), units.size() * sizeof(Unit));
    const int flags2[2] = {grad ? 1 : 0, ckpt};
    key = fnv1a(flags2, sizeof(flags2), key);
    key = fnv1a(&ctx->tune_epoch, sizeof(ctx->tune_epoch), key);

    if (!(ctx->plan.valid && ctx->plan.key == key)) {
        if (capturing(ctx))
            return fail(ctx, QAOA_ERR_INVALID,
                        "launch plan not built; run the same call once before stream capture");
        // ---- per-unit metadata: coefficients, tables, partials
        const int nu = (int)units.size();
        const int smax = small_max_n();
        std::vector<size_t> off_coef(nu), off_tab(nu), off_part(nu);
        std::vector<UnitLayout> lay(nu);
        size_t meta = 0;
        // coefficients of all units back to back (the sets of one eigenbasis
        // job are consecutive, so their rounds form a [set][round] array)
        std::vector<size_t> off_w(nu, 0);
        for (int i = 0; i < nu; i++) {
            off_coef[i] = meta;
            meta += sizeof(RoundCoef) * units[i].p * (units[i].ma ? units[i].n : (units[i].gm ? 2 : 1));
        }
        meta = align_up(meta);
        for (int i = 0; i < nu; i++) {
            const Unit &u = units[i];
            if (u.gm) {  // weight phases of the general X mixer, p x (n + 1)
                off_w[i] = meta;
                meta = align_up(meta + sizeof(float4) * u.p * (u.n + 1));
            }
            off_tab[i] = meta;
            if (u.cost_dtype == QAOA_COST_U8) meta = align_up(meta + sizeof(float2) * kPhaseTable * u.p);
            off_part[i] = meta;
            if (u.mixer_kind == QAOA_MIXER_X && u.n > smax) {
                lay[i] = layout_for(ctx, u, grad, ckpt);
                // partial slots: <C>, and with gradients every beta_k and gamma_k
                meta = align_up(meta + sizeof(double) * (grad ? 2 * u.p + 1 : 1) * lay[i].stride);
            }
        }
        void *d_meta = nullptr;
        qaoa_status st = scratch(ctx, "meta", meta, &d_meta);
        if (st) return st;
        char *mb = static_cast<char *>(d_meta);

        // ---- state memory: pass units grouped by launch shape, admitted in waves
        struct GKey {
            int Tf, Tb, Pf, Pb, p, dt, nbc, nbg, var;  // var: 0 X, 1 multi-angle, 2 general X mixer
            int fused;
            bool operator<(const GKey &o) const {
                return std::tie(Tf, Tb, Pf, Pb, p, dt, nbc, nbg, var, fused) <
                       std::tie(o.Tf, o.Tb, o.Pf, o.Pb, o.p, o.dt, o.nbc, o.nbg, o.var, o.fused);
            }
        };
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const size_t held = ctx->bufs.count("state") ? ctx->bufs["state"].bytes : 0;
        const double budget_d = (double)(free_b + held) * 0.92 - 1.0 * (1ull << 30);
        size_t budget = budget_d > 0 ? (size_t)budget_d : 0;
        if (ctx->state_limit >= 0) budget = std::min(budget, (size_t)ctx->state_limit);
        // fused round boundaries need per-pass checkpoints: a unit whose
        // checkpoints do not fit runs the unfused schedule (and may then step
        // down to fewer checkpoints below)
        for (int i = 0; i < nu; i++) {
            if (units[i].mixer_kind != QAOA_MIXER_X || units[i].n <= smax || !lay[i].fused || !grad) continue;
            if (align_up((size_t)lay[i].vecs * (sizeof(float2) << units[i].n)) > budget) {
                lay[i].fused = false;
                lay[i].vecs = layout_vecs(lay[i], units[i].p, grad);
            }
        }
        std::map<GKey, std::vector<int>> groups;
        for (int i = 0; i < nu; i++) {
            if (units[i].mixer_kind != QAOA_MIXER_X || units[i].n <= smax) continue;
            const UnitLayout &L = lay[i];
            groups[{L.T_f, L.T_b, (int)L.gf.size(), (int)L.gb.size(), units[i].p, units[i].cost_dtype, L.nb_bc,
                    L.nb_bg, units[i].ma ? 1 : (units[i].gm ? 2 : 0), L.fused ? L.fuse_mask : 0}]
                .push_back(i);
        }
        // waves: consecutive units of a group whose states fit the budget together
        struct Wave {
            GKey gk;
            std::vector<int> us;
            std::vector<size_t> soff;
        };
        std::vector<Wave> waves;
        size_t state_need = 0;
        for (auto &kv : groups) {
            Wave w;
            w.gk = kv.first;
            size_t used = 0;
            for (int i : kv.second) {
                size_t need = align_up((size_t)lay[i].vecs * (sizeof(float2) << units[i].n));
                // fewer checkpoints when one angle set's scratch does not fit
                while (need > budget && lay[i].ckpt > QAOA_CKPT_NONE && !units[i].gm) {
                    lay[i].ckpt--;
                    lay[i].vecs = layout_vecs(lay[i], units[i].p, grad);
                    need = align_up((size_t)lay[i].vecs * (sizeof(float2) << units[i].n));
                }
                if (need > budget)
                    return fail(ctx, QAOA_ERR_OOM,
                                "one angle set at n=%d needs %.2f GiB of state scratch, %.2f GiB available",
                                units[i].n, need / 1073741824.0, budget / 1073741824.0);
                if (used + need > budget && !w.us.empty()) {
                    waves.push_back(w);
                    w.us.clear();
                    w.soff.clear();
                    used = 0;
                }
                w.us.push_back(i);
                w.soff.push_back(used);
                used += need;
                state_need = std::max(state_need, used);
            }
            if (!w.us.empty()) waves.push_back(w);
        }
        void *d_state = nullptr;
        if (state_need) {
            st = scratch(ctx, "state", state_need, &d_state);
            if (st) return st;
        }

        // ---- descriptors
        std::vector<char> host;  // packed descriptor image
        auto put = [&](const void *src, size_t bytes) {
            const size_t off = align_up(host.size(), 16);
            host.resize(off + bytes);
            std::memcpy(host.data() + off, src, bytes);
            return off;
        };
        std::vector<LaunchRec> L;

        std::vector<PrepDesc> prep(nu);
        for (int i = 0; i < nu; i++) {
            const Unit &u = units[i];
            prep[i].angles = u.angles;
            prep[i].coef = reinterpret_cast<RoundCoef *>(mb + off_coef[i]);
            prep[i].table = u.cost_dtype == QAOA_COST_U8 ? reinterpret_cast<float2 *>(mb + off_tab[i]) : nullptr;
            prep[i].p = u.p;
            prep[i].tsize = u.tsize;
            prep[i].nq = u.ma ? u.n : 0;
            prep[i].gm_n = u.gm ? u.n : 0;
            prep[i].wts = u.gm ? u.wts : nullptr;
            prep[i].wtab = u.gm ? reinterpret_cast<float4 *>(mb + off_w[i]) : nullptr;
        }
        {
            // the n = 12 tile kernel forms its coefficients itself
            std::vector<PrepDesc> todo;
            for (int i = 0; i < nu; i++) {
                const Unit &u = units[i];
                if (!(u.mixer_kind == QAOA_MIXER_X && u.n == kPassTileBits && !u.ma && !u.gm)) todo.push_back(prep[i]);
            }
            if (!todo.empty()) {
                LaunchRec r;
                r.kind = LK_PREP;
                r.desc_off = put(todo.data(), sizeof(PrepDesc) * todo.size());
                r.ndesc = (int)todo.size();
                r.fam = family(ctx, "prep_coefficients");
                L.push_back(r);
            }
        }
        // on-chip units: n = 12 with the transverse field as one register-staged
        // tile (t12), every other n <= 12 unit in the generic kernel
        for (int combo = 0; combo < 4; combo++) {
            const int dt = combo & 1, t12 = combo >> 1;
            std::vector<SmallDesc> sd;
            int maxn = 0;
            double bytes = 0;
            for (int i = 0; i < nu; i++) {
                const Unit &u = units[i];
                if (u.mixer_kind != QAOA_MIXER_X || u.n > smax || u.cost_dtype != dt) continue;
                if ((u.n == kPassTileBits && !u.ma && !u.gm) != (t12 != 0)) continue;
                SmallDesc s;
                std::memset(&s, 0, sizeof(s));
                s.cost = u.cost;
                s.init = u.init;
                s.coef = prep[i].coef;
                s.table = prep[i].table;
                s.E_out = u.E;
                s.grad_out = grad ? u.grad : nullptr;
                s.n = u.n;
                s.p = u.p;
                s.nq = u.ma ? u.n : 0;
                s.wts = u.gm ? u.wts : nullptr;
                s.angles_beta = u.angles;
                s.amp0 = 1.0f / std::sqrt((float)(1u << u.n));
                sd.push_back(s);
                maxn = std::max(maxn, u.n);
                bytes += std::ldexp(1.0, u.n) * (dt == QAOA_COST_U8 ? 1 : 4) * (grad ? 3 : 2);
            }
            if (sd.empty()) continue;
            LaunchRec r;
            r.kind = LK_SMALL;
            r.cost_dtype = dt;
            r.desc_off = put(sd.data(), sizeof(SmallDesc) * sd.size());
            r.ndesc = (int)sd.size();
            r.small_maxn = maxn;
            r.small_grad = grad ? 1 : 0;
            r.t12 = t12;
            r.bytes = bytes;
            r.fam = family(ctx, std::string(t12 ? "tile12_" : "small_") + (grad ? "grad_" : "fwd_") + dtype_name(dt));
            L.push_back(r);
        }
        std::vector<RedChunk> rchunks;
        std::vector<RedOut> routs;
        size_t level2_need = 0;  // chunks of the largest reduction launch
        // partials of unit quantity q: cnt values at src -> chunks + one output
        auto add_reduction_to = [&](std::vector<RedChunk> &chunks, std::vector<RedOut> &outs, const double *src,
                                    int64_t cnt, double *out, double scale) {
            RedOut o;
            o.first = (int)chunks.size();
            for (int64_t j = 0; j < cnt; j += kRedChunk) {
                RedChunk ch;
                ch.src = src + j;
                ch.cnt = (int)std::min<int64_t>(kRedChunk, cnt - j);
                ch.pad = 0;
                chunks.push_back(ch);
            }
            o.n = (int)chunks.size() - o.first;
            o.out = out;
            o.scale = scale;
            outs.push_back(o);
        };
        auto add_reduction = [&](const double *src, int64_t cnt, double *out, double scale) {
            add_reduction_to(rchunks, routs, src, cnt, out, scale);
        };
        // tensor maps of gathered tiles with short runs (< 2^kTmaSegBits elements),
        // deduplicated; PassDesc.tm_* temporarily hold (index + 1)
        std::vector<CUtensorMap> maps;
        std::map<std::tuple<const void *, int, int, int, int>, size_t> map_index;
        std::vector<std::pair<size_t, int>> xpass_descs;  // (image offset, count)
        int n_sched = 0;
        bool any_eig_tc = false;
        auto map_for = [&](const void *basep, int n, int c, int lo, int elsz) -> const void * {
            const auto key = std::make_tuple(basep, n, c, lo, elsz);
            auto it = map_index.find(key);
            size_t idx;
            if (it != map_index.end()) {
                idx = it->second;
            } else {
                CUtensorMap m;
                if (!encode_gather_map(&m, basep, n, c, lo, elsz)) return nullptr;
                idx = maps.size();
                maps.push_back(m);
                map_index[key] = idx;
            }
            return reinterpret_cast<const void *>((uintptr_t)(idx + 1));
        };
        auto attach_maps = [&](PassDesc &d, bool bwd, int dt) {
            if (d.c >= kTmaSegBits) return;
            const int lo = d.gpos[d.c];
            const int cb = dt == QAOA_COST_U8 ? 1 : 4;
            const bool ld_psi = bwd || !(d.flags & PF_GEN_INIT);
            const bool ld_lam = bwd && !(d.flags & PF_LAM_FROM_C);
            const bool ld_cost = bwd ? (d.flags & (PF_LAM_FROM_C | PF_PHASE | PF_FUSED))
                                     : (d.flags & (PF_PHASE | PF_E | PF_FUSED));
            if (ld_psi) d.tm_psi = map_for(d.psi_in, d.n, d.c, lo, 8);
            if (ld_lam) d.tm_lam = map_for(d.lam_in, d.n, d.c, lo, 8);
            if (ld_cost) d.tm_cost = map_for(d.cost, d.n, d.c, lo, cb);
        };
        for (const Wave &w : waves) {
            const GKey &gk = w.gk;
            std::vector<std::vector<PassDesc>> steps;
            // <C> of every unit of the wave, reduced between the forward and
            // the adjoint sweep: the adjoint shifts the cost by it
            std::vector<RedChunk> mchunks;
            std::vector<RedOut> mouts;
            for (size_t wi = 0; wi < w.us.size(); wi++) {
                const int i = w.us[wi];
                const Unit &u = units[i];
                const int64_t N = 1ll << u.n;
                float2 *base = reinterpret_cast<float2 *>(static_cast<char *>(d_state) + w.soff[wi]);
                float2 *W = base, *Lam = grad ? base + N : nullptr, *CK = grad ? base + 2 * N : nullptr;
                if (grad && lay[i].ckpt == QAOA_CKPT_PASS) {
                    Lam = base;
                    CK = base + N;
                    W = nullptr;
                }
                std::vector<PassDesc> f, b;
                unit_passes(u, lay[i], grad, W, Lam, CK, prep[i].coef, prep[i].table, prep[i].wtab,
                            reinterpret_cast<double *>(mb + off_part[i]), f, b);
                for (PassDesc &d : b) d.c0 = u.E;
                std::vector<PassDesc> all = f;
                all.insert(all.end(), b.begin(), b.end());
                if (steps.size() < all.size()) steps.resize(all.size());
                for (size_t s = 0; s < all.size(); s++) steps[s].push_back(all[s]);
                {
                    const double *part = reinterpret_cast<const double *>(mb + off_part[i]);
                    const int64_t S = lay[i].stride;
                    if (grad)
                        add_reduction_to(mchunks, mouts, part, (int64_t)lay[i].tiles_f * kPassWarps, u.E, 1.0);
                    else
                        add_reduction(part, (int64_t)lay[i].tiles_f * kPassWarps, u.E, 1.0);
                    if (grad) {
                        const int64_t tw = (int64_t)lay[i].tiles_b * kPassWarps;
                        const int Pb = (int)lay[i].gb.size();
                        const int nbq = u.ma ? u.n : 1;
                        for (int k = 0; k < u.p; k++) {
                            if (u.gm) {  // the weight-diagonal pass holds the whole beta partial
                                add_reduction(part + (1 + k) * S, tw, u.grad + k, 2.0);
                            } else if (u.ma) {
                                // qubit of local bit j in adjoint pass q (group Pb - 1 - q)
                                for (int q = 0; q < Pb; q++) {
                                    const Group &G = lay[i].gb[Pb - 1 - q];
                                    for (int j = (G.c >= kPassTileBits ? 0 : G.c); j < kPassTileBits; j++) {
                                        const int qb = G.c >= kPassTileBits ? j : G.lo + (j - G.c);
                                        add_reduction(part + (1 + k) * S + ((int64_t)q * kPassTileBits + j) * tw, tw,
                                                      u.grad + (int64_t)k * u.n + qb, 2.0);
                                    }
                                }
                            } else {
                                add_reduction(part + (1 + k) * S, (int64_t)Pb * tw, u.grad + k, 2.0);
                            }
                            add_reduction(part + (1 + u.p + k) * S, tw, u.grad + (int64_t)u.p * nbq + k, 2.0);
                        }
                    }
                }
            }
            const int nfwd = forward_passes(lay[w.us[0]], gk.p);
            for (size_t s = 0; s < steps.size(); s++) {
                const bool bwd = (int)s >= nfwd;
                const int T = bwd ? gk.Tb : gk.Tf;
                std::vector<uint32_t> tb(steps[s].size() + 1, 0);
                double bytes = 0;
                for (size_t j = 0; j < steps[s].size(); j++) {
                    tb[j + 1] = tb[j] + steps[s][j].ntiles;
                    bytes += pass_bytes(steps[s][j], bwd, gk.dt == QAOA_COST_U8 ? 1 : 4);
                    attach_maps(steps[s][j], bwd, gk.dt);
                }
                LaunchRec r;
                r.kind = LK_XPASS;
                r.T = T;
                r.bwd = bwd;
                r.cost_dtype = gk.dt;
                r.nbuf = bwd ? (steps[s][0].c >= kPassTileBits ? gk.nbc : gk.nbg) : 2;
                // round-boundary adjoint passes: one buffer and two CTAs per SM
                // (measured at n = 28: 2.72 ms a launch against 3.22 with two
                // buffers and one CTA; they are bound by SM latency, not loads)
                if (bwd && (steps[s][0].flags & PF_FUSED)) r.nbuf = fused_bwd_nbuf();
                r.var = gk.var;
                r.desc_off = put(steps[s].data(), sizeof(PassDesc) * steps[s].size());
                xpass_descs.push_back({r.desc_off, (int)steps[s].size()});
                r.tb_off = put(tb.data(), sizeof(uint32_t) * tb.size());
                r.ndesc = (int)steps[s].size();
                r.tiles = tb.back();
                r.bytes = bytes;
                r.sched_idx = n_sched++;
                r.fused = (steps[s][0].flags & PF_FUSED) ? 1 : 0;
                {
                    const uint32_t cost_flags =
                        bwd ? (PF_LAM_FROM_C | PF_PHASE | PF_FUSED) : (PF_PHASE | PF_E | PF_FUSED);
                    r.cost_free = 1;
                    for (const PassDesc &pd : steps[s])
                        if (pd.flags & cost_flags) r.cost_free = 0;
                }
                char nm[64];
                const int c0 = steps[s][0].c;
                snprintf(nm, sizeof(nm), "xpass%s_%s%s_%s_%s", gk.var == 1 ? "_ma" : (gk.var == 2 ? "_gm" : ""),
                         bwd ? "bwd" : "fwd", (steps[s][0].flags & PF_FUSED) ? "_fused" : "",
                         c0 >= kPassTileBits ? "contig" : (c0 >= 6 ? "gather_wide" : "gather"),
                         dtype_name(gk.dt));
                r.fam = family(ctx, nm);
                L.push_back(r);
                if (grad && (int)s == nfwd - 1 && !mouts.empty()) {
                    LaunchRec m;
                    m.kind = LK_REDUCE;
                    m.desc_off = put(mchunks.data(), sizeof(RedChunk) * mchunks.size());
                    m.tb_off = put(mouts.data(), sizeof(RedOut) * mouts.size());
                    m.ndesc = (int)mchunks.size();
                    m.tiles = (uint32_t)mouts.size();
                    m.fam = family(ctx, "reduce_expectation");
                    level2_need = std::max(level2_need, mchunks.size());
                    L.push_back(m);
                }
            }
        }
        // ---- Grover-mixer units: the rank-one update as streaming passes, one
        // launch per pass over all units of one (p, cost dtype), admitted in
        // waves under the memory left next to the X-mixer states
        {
            std::map<std::pair<int, int>, std::vector<int>> rgroups;
            for (int i = 0; i < nu; i++)
                if (units[i].mixer_kind == QAOA_MIXER_GROVER)
                    rgroups[{units[i].p, units[i].cost_dtype}].push_back(i);
            if (!rgroups.empty()) {
                const int64_t tile = r1_tile_amps();
                const uint32_t gmax = r1_max_grid();
                const size_t held_r1 = ctx->bufs.count("r1state") ? ctx->bufs["r1state"].bytes : 0;
                const double rb = (double)(free_b + held + held_r1) * 0.92 - 1.0 * (1ull << 30);
                size_t r1_budget = rb > 0 ? (size_t)rb : 0;
                if (ctx->state_limit >= 0) r1_budget = std::min(r1_budget, (size_t)ctx->state_limit);
                r1_budget = r1_budget > state_need ? r1_budget - state_need : 0;
                struct RUnit {
                    int i;
                    int64_t ld;
                    int ck;
                    uint32_t nt;
                    size_t soff, part_off, scal_off;
                };
                struct RWave {
                    int p, dt;
                    std::vector<RUnit> us;
                };
                std::vector<RWave> rwaves;
                size_t r1_need = 0, r1_meta = 0;
                for (auto &kv : rgroups) {
                    RWave w;
                    w.p = kv.first.first;
                    w.dt = kv.first.second;
                    size_t used = 0;
                    uint64_t wtiles = 0;
                    for (int i : kv.second) {
                        const Unit &u = units[i];
                        RUnit ru;
                        ru.i = i;
                        ru.ld = (u.dim + 63) / 64 * 64;
                        ru.nt = (uint32_t)((u.dim + tile - 1) / tile);
                        const size_t vb = (size_t)ru.ld * sizeof(float2);
                        // p + 1 vectors (phi_0..phi_{p-1} and lambda) with checkpoints,
                        // else phi and lambda, the adjoint undoing each round on phi
                        ru.ck = grad && ckpt != QAOA_CKPT_NONE ? 1 : 0;
                        size_t need = align_up(vb * (grad ? (ru.ck ? u.p + 1 : 2) : 1));
                        if (need > r1_budget && ru.ck) {
                            ru.ck = 0;
                            need = align_up(vb * 2);
                        }
                        if (need > r1_budget)
                            return fail(ctx, QAOA_ERR_OOM,
                                        "one Grover-mixer angle set of %lld states needs %.2f GiB of state scratch, "
                                        "%.2f GiB available",
                                        (long long)u.dim, need / 1073741824.0, r1_budget / 1073741824.0);
                        if (!w.us.empty() && (used + need > r1_budget || wtiles + ru.nt >= (1ull << 31))) {
                            rwaves.push_back(w);
                            w.us.clear();
                            used = 0;
                            wtiles = 0;
                        }
                        ru.soff = used;
                        used += need;
                        wtiles += ru.nt;
                        ru.part_off = r1_meta;
                        r1_meta = align_up(r1_meta + sizeof(double) * 3 * std::min<uint32_t>(ru.nt, gmax));
                        ru.scal_off = r1_meta;
                        r1_meta = align_up(r1_meta + sizeof(double) * (4 * u.p + 3));
                        w.us.push_back(ru);
                        r1_need = std::max(r1_need, used);
                    }
                    if (!w.us.empty()) rwaves.push_back(w);
                }
                void *d_r1 = nullptr, *d_r1m = nullptr;
                st = scratch(ctx, "r1state", r1_need, &d_r1);
                if (st) return st;
                st = scratch(ctx, "r1meta", r1_meta, &d_r1m);
                if (st) return st;
                for (const RWave &w : rwaves) {
                    std::vector<R1Desc> ds;
                    std::vector<uint32_t> tb(1, 0);
                    for (const RUnit &ru : w.us) {
                        const Unit &u = units[ru.i];
                        R1Desc d;
                        std::memset(&d, 0, sizeof(d));
                        d.cost = u.cost;
                        d.init = u.init;
                        d.coef = prep[ru.i].coef;
                        d.table = prep[ru.i].table;
                        d.angles = u.angles;
                        float2 *base = reinterpret_cast<float2 *>(static_cast<char *>(d_r1) + ru.soff);
                        d.phi = base;
                        d.lam = grad ? base + (ru.ck ? (int64_t)u.p * ru.ld : ru.ld) : nullptr;
                        d.part = reinterpret_cast<double *>(static_cast<char *>(d_r1m) + ru.part_off);
                        d.scal = reinterpret_cast<double *>(static_cast<char *>(d_r1m) + ru.scal_off);
                        d.E = u.E;
                        d.grad = grad ? u.grad : nullptr;
                        d.dim = u.dim;
                        d.ld = ru.ld;
                        d.p = u.p;
                        d.ckpt = ru.ck;
                        d.amp0 = (float)(1.0 / std::sqrt((double)u.dim));
                        ds.push_back(d);
                        tb.push_back(tb.back() + ru.nt);
                    }
                    const size_t doff = put(ds.data(), sizeof(R1Desc) * ds.size());
                    const size_t toff = put(tb.data(), sizeof(uint32_t) * tb.size());
                    const double cb = w.dt == QAOA_COST_U8 ? 1.0 : 4.0;
                    // algorithmic bytes of one pass over every unit of the wave
                    auto pass_bytes_r1 = [&](int mode, int round) {
                        double b = 0;
                        for (const RUnit &ru : w.us) {
                            const Unit &u = units[ru.i];
                            const double N = (double)u.dim;
                            double per = cb;  // the cost value
                            if (mode == R1_FWD) per += (round == 0 && !u.init) ? 8 : 16;
                            else if (mode == R1_LAST) per += 8;
                            else {
                                per += 8 + (round == w.p - 1 ? 0 : 8);  // phi, lambda
                                if (round > 0) per += 8 + (ru.ck ? 0 : 8);  // lambda (and phi) out
                            }
                            b += N * per;
                        }
                        return b;
                    };
                    const char *mname[3] = {"fwd", "last", "bwd"};
                    auto add = [&](int mode, int round) {
                        LaunchRec r;
                        r.kind = LK_R1_PASS;
                        r.cost_dtype = w.dt;
                        r.desc_off = doff;
                        r.tb_off = toff;
                        r.ndesc = (int)ds.size();
                        r.tiles = tb.back();
                        r.r1mode = mode;
                        r.r1round = round;
                        r.r1grid = std::min<uint32_t>(tb.back(), r1_grid(mode, w.dt));
                        r.bytes = pass_bytes_r1(mode, round);
                        char nm[48];
                        snprintf(nm, sizeof(nm), "grover_r1_%s_%s", mname[mode], dtype_name(w.dt));
                        r.fam = family(ctx, nm);
                        L.push_back(r);
                        LaunchRec q;
                        q.kind = LK_R1_SCALAR;
                        q.desc_off = doff;
                        q.tb_off = toff;
                        q.ndesc = (int)ds.size();
                        q.r1mode = mode == R1_FWD ? R1_SFWD : (mode == R1_LAST ? R1_SLAST : R1_SBWD);
                        q.r1round = round;
                        q.r1grid = r.r1grid;
                        q.fam = family(ctx, "grover_r1_scalar");
                        L.push_back(q);
                    };
                    for (int k = 0; k < w.p; k++) add(R1_FWD, k);
                    add(R1_LAST, w.p - 1);
                    if (grad)
                        for (int k = w.p - 1; k >= 0; k--) add(R1_BWD, k);
                }
            }
        }
        // ---- eigenbasis-mixer jobs: one GEMM pipeline per job, the job's angle
        // sets as the columns of every product
        {
            struct EG {
                int u0, S, Spad, ld, nmt;
                size_t st_off, part_off, c0_off;
                bool sym;
                const SymLayout *L;
                int nob;  // orbit blocks (block-diagonal mixers)
            };
            std::vector<EG> eg;
            size_t st_bytes = 0, part_bytes = 0;
            auto is_eig = [](int kind) { return kind == QAOA_MIXER_EIGEN || kind == QAOA_MIXER_EIGEN_SYM; };
            for (int i = 0; i < nu;) {
                if (!is_eig(units[i].mixer_kind)) {
                    i++;
                    continue;
                }
                int j = i;
                while (j < nu && units[j].mixer_kind == units[i].mixer_kind && units[j].job == units[i].job) j++;
                const Unit &u = units[i];
                if (u.gemm_precision == QAOA_GEMM_BF16X3)
                    return fail(ctx, QAOA_ERR_UNSUPPORTED,
                                "BF16x3 products (16-bit split, ~1e-5 relative) cannot meet the 1e-5 tolerance; "
                                "use QAOA_GEMM_3XTF32");
                EG g;
                g.u0 = i;
                g.S = j - i;
                g.Spad = (int)align_up((size_t)g.S, kEigSetTile);
                g.sym = u.mixer_kind == QAOA_MIXER_EIGEN_SYM;
                g.L = nullptr;
                g.nob = 0;
                if (g.sym) {
                    auto key = std::make_pair(u.n, u.k);
                    if (!ctx->sym.count(key)) {
                        SymLayout SL;
                        if (!build_sym_layout(u.n, u.k, SL))
                            return fail(ctx, QAOA_ERR_INVALID, "no cyclic-shift layout for n=%d, k=%d", u.n, u.k);
                        ctx->sym[key] = SL;
                    }
                    g.L = &ctx->sym[key];
                    g.ld = g.L->ldp;
                    g.nob = (g.L->n_orbits + kOrbitsPerBlock - 1) / kOrbitsPerBlock;
                } else {
                    g.ld = (int)align_up((size_t)u.dim, kEigTile);
                }
                g.nmt = g.ld / kEigTile;
                const size_t mat = (size_t)2 * g.Spad * g.ld * sizeof(float);
                const int tcp = u.gemm_precision == QAOA_GEMM_3XTF32 ? 1 : 0;
                // dense: X, Y, L (+ their remainder planes on the tensor-core path) and 2p
                // checkpoints; block-diagonal: one more work matrix Z (product outputs
                // that only the orbit kernel reads)
                const int nmat = (grad ? 3 + 2 * u.p + 3 * tcp : 2 + 2 * tcp) + (g.sym ? 1 : 0);
                g.st_off = st_bytes;
                st_bytes += align_up(mat * nmat);
                g.part_off = part_bytes;
                part_bytes += align_up(sizeof(double) * (1 + 2 * u.p) * g.Spad * std::max(g.nmt, g.nob));
                g.c0_off = part_bytes;  // the job's cost mean (shift of the adjoint)
                part_bytes += align_up(sizeof(double));
                eg.push_back(g);
                i = j;
            }
            if (!eg.empty()) {
                if (ctx->state_limit >= 0 && st_bytes > (size_t)ctx->state_limit)
                    return fail(ctx, QAOA_ERR_OOM,
                                "eigenbasis state matrices need %.3f GiB, the context's limit is %.3f GiB",
                                st_bytes / 1073741824.0, ctx->state_limit / 1073741824.0);
                void *d_est = nullptr, *d_epart = nullptr;
                st = scratch(ctx, "eigstate", st_bytes, &d_est);
                if (st) return st;
                st = scratch(ctx, "eigpart", part_bytes, &d_epart);
                if (st) return st;
                for (const EG &g : eg) {
                    const Unit &u = units[g.u0];
                    if (g.sym) {
                        st = plan_sym_job(ctx, units, g.u0, g.S, g.Spad, grad, *g.L, g.nmt, g.nob,
                                          static_cast<char *>(d_est) + g.st_off,
                                          reinterpret_cast<double *>(static_cast<char *>(d_epart) + g.part_off),
                                          reinterpret_cast<double *>(static_cast<char *>(d_epart) + g.c0_off),
                                          reinterpret_cast<const RoundCoef *>(mb + off_coef[g.u0]), L, add_reduction,
                                          any_eig_tc);
                        if (st) return st;
                        continue;
                    }
                    const int D = (int)u.dim, ld = g.ld, p = u.p;
                    // padded V, V^T and split eigenvalues, prepared once per (V, lambda)
                    const bool tcp = u.gemm_precision == QAOA_GEMM_3XTF32;
                    char nm[96];
                    void *dV = nullptr, *dVt = nullptr, *dL = nullptr, *dVl = nullptr, *dVtl = nullptr;
                    // operand planes: kept across calls for a mixer the caller gave an id
                    // (the id promises V and lambda do not change), else rebuilt by
                    // every call from the V and lambda it is given
                    if (u.mixer_id)
                        snprintf(nm, sizeof(nm), "eigV:id%llu:%d:%d", (unsigned long long)u.mixer_id, D, tcp ? 1 : 0);
                    else
                        snprintf(nm, sizeof(nm), "eigV:call:%d:%d", D, tcp ? 1 : 0);
                    const std::string key = nm;
                    st = scratch(ctx, (key + ":V").c_str(), (size_t)ld * ld * sizeof(float), &dV);
                    if (st) return st;
                    st = scratch(ctx, (key + ":Vt").c_str(), (size_t)ld * ld * sizeof(float), &dVt);
                    if (st) return st;
                    if (tcp) {
                        st = scratch(ctx, (key + ":Vlo").c_str(), (size_t)ld * ld * sizeof(float), &dVl);
                        if (st) return st;
                        st = scratch(ctx, (key + ":Vtlo").c_str(), (size_t)ld * ld * sizeof(float), &dVtl);
                        if (st) return st;
                    }
                    st = scratch(ctx, (key + ":lam").c_str(), (size_t)2 * ld * sizeof(float), &dL);
                    if (st) return st;
                    if (!u.mixer_id || !ctx->eig_ready.count(key)) {
                        LaunchRec r;
                        r.kind = LK_OPERANDS;
                        r.op.sym = 0;
                        r.op.V = u.V;
                        r.op.lam = u.lam;
                        r.op.D = D;
                        r.op.ld = ld;
                        r.op.Vp = static_cast<float *>(dV);
                        r.op.Vtp = static_cast<float *>(dVt);
                        r.op.Vpl = static_cast<float *>(dVl);
                        r.op.Vtpl = static_cast<float *>(dVtl);
                        r.op.lam_hi = static_cast<float *>(dL);
                        r.op.lam_lo = static_cast<float *>(dL) + ld;
                        r.fam = family(ctx, "eig_operands");
                        if (u.mixer_id) {  // once for this mixer, now
                            st = launch_operands(ctx, r);
                            if (st) return st;
                            ctx->eig_ready.insert(key);
                        } else {
                            L.push_back(r);
                        }
                    }
                    const float *Vp = static_cast<const float *>(dV), *Vtp = static_cast<const float *>(dVt);
                    const float *lam_hi = static_cast<const float *>(dL), *lam_lo = lam_hi + ld;
                    const size_t mat = (size_t)2 * g.Spad * ld;
                    float *base = reinterpret_cast<float *>(static_cast<char *>(d_est) + g.st_off);
                    float *X = base, *Y = base + mat, *Lm = grad ? base + 2 * mat : nullptr;
                    auto CKX = [&](int k) { return base + (3 + k) * mat; };
                    auto CKY = [&](int k) { return base + (3 + p + k) * mat; };
                    // remainder planes (tensor-core path) after everything else
                    const int lo0 = grad ? 3 + 2 * p : 2;
                    float *Xl = tcp ? base + lo0 * mat : nullptr;
                    float *Yl = tcp ? base + (lo0 + 1) * mat : nullptr;
                    float *Ll = (tcp && grad) ? base + (lo0 + 2) * mat : nullptr;
                    const float *Vpl = static_cast<const float *>(dVl), *Vtpl = static_cast<const float *>(dVtl);
                    double *part = reinterpret_cast<double *>(static_cast<char *>(d_epart) + g.part_off);
                    const int64_t pq = (int64_t)g.Spad * g.nmt;  // partials per quantity
                    const RoundCoef *coef = reinterpret_cast<const RoundCoef *>(mb + off_coef[g.u0]);
                    EigEpiParams ep{};
                    ep.M = D;
                    ep.ld = ld;
                    ep.nsets = g.S;
                    ep.lam_hi = lam_hi;
                    ep.lam_lo = lam_lo;
                    ep.cost = u.cost;
                    ep.cost_dtype = u.cost_dtype;
                    ep.coef = coef;
                    ep.coef_stride = p;
                    ep.part_stride = g.nmt;
                    double *c0 = reinterpret_cast<double *>(static_cast<char *>(d_epart) + g.c0_off);
                    ep.c0 = grad ? c0 : nullptr;
                    if (grad) {
                        LaunchRec r;
                        r.kind = LK_COST_MEAN;
                        r.ep = ep;
                        r.mean_out = c0;
                        r.fam = family(ctx, "cost_mean");
                        L.push_back(r);
                    }
                    const double gflops = 2.0 * D * (double)D * 2.0 * g.S;
                    const int fam_g = family(ctx, tcp ? "eig_gemm_tc_3xtf32" : "eig_gemm_simt");
                    // B operand planes of each state matrix (hi = the matrix itself on the tensor path)
                    auto lo_of = [&](const float *B) -> const float * {
                        return B == X ? Xl : B == Y ? Yl : B == Lm ? Ll : nullptr;
                    };
                    bool map_ok = true;
                    auto gemm = [&](const float *A, const float *B, EigEpiParams q) {
                        LaunchRec r;
                        r.kind = LK_EIG_GEMM;
                        r.gA = A;
                        r.gB = B;
                        r.Mp = ld;
                        r.Np = 2 * g.Spad;
                        r.Kp = ld;
                        r.flops = gflops;
                        r.fam = fam_g;
                        if (tcp) {
                            r.tc = 1;
                            any_eig_tc = true;
                            const float *Al = A == Vp ? Vpl : Vtpl;
                            map_ok = map_ok && encode_kmajor_map(&r.tm[0], A, ld, ld) &&
                                     encode_kmajor_map(&r.tm[1], Al, ld, ld) &&
                                     encode_kmajor_map(&r.tm[2], B, ld, 2 * g.Spad) &&
                                     encode_kmajor_map(&r.tm[3], lo_of(B), ld, 2 * g.Spad);
                            // outputs that feed the next product carry their remainder plane
                            q.out_lo = q.out == X ? Xl : q.out == Y ? Yl : q.out == Lm ? Ll : nullptr;
                            q.out2_lo = q.out2 == Lm ? Ll : nullptr;
                            if (q.kind == EPI_FWD_LAST) q.out_lo = nullptr;  // psi_p is not a product operand
                        }
                        r.ep = q;
                        L.push_back(r);
                    };
                    {
                        LaunchRec r;
                        r.kind = LK_EIG_INIT;
                        r.ep = ep;
                        r.iX = X;
                        r.iX_lo = Xl;
                        r.ick0 = grad ? CKX(0) : nullptr;
                        r.iinit = u.init;
                        r.iamp0 = (float)(1.0 / std::sqrt((double)D));
                        r.fam = family(ctx, "eig_init");
                        L.push_back(r);
                    }
                    for (int k = 0; k < p; k++) {
                        EigEpiParams q = ep;
                        q.kind = EPI_FWD_EIG;
                        q.round = k;
                        q.out = Y;
                        q.ckpt = grad ? CKY(k) : nullptr;
                        gemm(Vtp, X, q);
                        q = ep;
                        if (k < p - 1) {
                            q.kind = EPI_FWD_PHASE;
                            q.round = k + 1;
                            q.out = X;
                            q.ckpt = grad ? CKX(k + 1) : nullptr;
                        } else {
                            q.kind = EPI_FWD_LAST;
                            q.round = k;
                            q.out = grad ? X : nullptr;
                            q.out2 = Lm;
                            q.part = part;
                        }
                        gemm(Vp, Y, q);
                    }
                    if (grad) {
                        for (int k = p - 1; k >= 0; k--) {
                            EigEpiParams q = ep;
                            q.kind = EPI_BWD_EIG;
                            q.round = k;
                            q.out = Y;
                            q.ck_in = CKY(k);
                            q.part = part + (1 + k) * pq;
                            gemm(Vtp, Lm, q);
                            q = ep;
                            q.kind = EPI_BWD_PHASE;
                            q.round = k;
                            q.out = k > 0 ? Lm : nullptr;
                            q.ck_in = CKX(k);
                            q.part = part + (1 + p + k) * pq;
                            gemm(Vp, Y, q);
                        }
                    }
                    if (!map_ok) return fail(ctx, QAOA_ERR_CUDA, "tensor map encoding failed");
                    for (int s2 = 0; s2 < g.S; s2++) {
                        const Unit &us = units[g.u0 + s2];
                        add_reduction(part + (int64_t)s2 * g.nmt, g.nmt, us.E, 1.0);
                        if (grad)
                            for (int k = 0; k < p; k++) {
                                add_reduction(part + (1 + k) * pq + (int64_t)s2 * g.nmt, g.nmt, us.grad + k, 2.0);
                                add_reduction(part + (1 + p + k) * pq + (int64_t)s2 * g.nmt, g.nmt,
                                              us.grad + p + k, 2.0);
                            }
                    }
                }
            }
        }
        if (!routs.empty()) {
            LaunchRec r;
            r.kind = LK_REDUCE;
            r.desc_off = put(rchunks.data(), sizeof(RedChunk) * rchunks.size());
            r.tb_off = put(routs.data(), sizeof(RedOut) * routs.size());
            r.ndesc = (int)rchunks.size();
            r.tiles = (uint32_t)routs.size();
            r.fam = family(ctx, "reduce_partials");
            L.push_back(r);
        }
        level2_need = std::max(level2_need, rchunks.size());
        if (level2_need) {
            void *d_l2 = nullptr;
            st = scratch(ctx, "level2", sizeof(double) * level2_need, &d_l2);
            if (st) return st;
        }
        // ---- tensor maps at the end of the image (128-byte aligned), then
        // the device addresses patched into the descriptors
        size_t maps_off = 0;
        if (!maps.empty()) {
            maps_off = align_up(host.size(), 128);
            host.resize(maps_off + maps.size() * sizeof(CUtensorMap));
            std::memcpy(host.data() + maps_off, maps.data(), maps.size() * sizeof(CUtensorMap));
        }
        // ---- upload
        void *d_desc = nullptr;
        st = scratch(ctx, "desc", host.size(), &d_desc);
        if (st) return st;
        for (const auto &xd : xpass_descs) {
            PassDesc *pd = reinterpret_cast<PassDesc *>(host.data() + xd.first);
            for (int j = 0; j < xd.second; j++) {
                const void **fields[3] = {&pd[j].tm_psi, &pd[j].tm_lam, &pd[j].tm_cost};
                for (const void **f : fields)
                    if (*f)
                        *f = static_cast<char *>(d_desc) + maps_off +
                             ((uintptr_t)*f - 1) * sizeof(CUtensorMap);
            }
        }
        st = host_stage(ctx, host.size());
        if (st) return st;
        std::memcpy(ctx->h_stage, host.data(), host.size());
        QG_CUDA(ctx, cudaMemcpyAsync(d_desc, ctx->h_stage, host.size(), cudaMemcpyHostToDevice, ctx->stream),
                "descriptor upload");
        QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "descriptor upload");
        if (n_sched > 0) {
            void *d_sched = nullptr;
            st = scratch(ctx, "sched", sizeof(uint32_t) * n_sched, &d_sched);
            if (st) return st;
        }
        if (any_eig_tc) {
            void *d_split = nullptr;
            st = scratch(ctx, "eig_split", eig_split_bytes(), &d_split);
            if (st) return st;
        }
        ctx->plan.launches = L;
        ctx->plan.n_sched = n_sched;
        ctx->plan.eig_tc = any_eig_tc;
        ctx->plan.key = key;
        ctx->plan.valid = true;
    }

    // ---- enqueue
    char *db = static_cast<char *>(ctx->bufs["desc"].p);
    uint32_t *d_sched = nullptr;
    if (ctx->plan.n_sched > 0) {
        d_sched = static_cast<uint32_t *>(ctx->bufs["sched"].p);
        QG_CUDA(ctx, cudaMemsetAsync(d_sched, 0, sizeof(uint32_t) * ctx->plan.n_sched, ctx->stream),
                "tile counters clear");
    }
    float *d_split_ws = nullptr;
    unsigned *d_split_cnt = nullptr;
    if (ctx->plan.eig_tc) {
        char *b = static_cast<char *>(ctx->bufs["eig_split"].p);
        d_split_cnt = reinterpret_cast<unsigned *>(b);
        d_split_ws = reinterpret_cast<float *>(b + eig_split_cnt_bytes());
        QG_CUDA(ctx, cudaMemsetAsync(d_split_cnt, 0, eig_split_cnt_bytes(), ctx->stream), "split counters clear");
    }
    const bool prof = ctx->profiling && !capturing(ctx);
    for (const LaunchRec &r : ctx->plan.launches) {
        NvtxRange nvtx_launch(r.fam >= 0 && r.fam < (int)ctx->fam_names.size() ? ctx->fam_names[r.fam].c_str()
                                                                              : "qaoa_launch");
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (prof) {
            ea = take_event(ctx);
            eb = take_event(ctx);
            cudaEventRecord(ea, ctx->stream);
        }
        cudaError_t e = cudaSuccess;
        switch (r.kind) {
        case LK_PREP:
            e = launch_prep(reinterpret_cast<const PrepDesc *>(db + r.desc_off), r.ndesc, ctx->d_err,
                            ctx->stream);
            break;
        case LK_SMALL:
            if (r.t12)
                e = launch_tile12(reinterpret_cast<const SmallDesc *>(db + r.desc_off), r.ndesc, r.cost_dtype,
                                  r.small_grad, ctx->d_err, ctx->stream);
            else
                e = launch_small(reinterpret_cast<const SmallDesc *>(db + r.desc_off), r.ndesc, r.cost_dtype,
                                 r.small_grad, r.small_maxn, ctx->d_err, ctx->stream);
            break;
        case LK_XPASS:
            e = launch_xpass(r.bwd, r.cost_dtype, r.nbuf, r.var, reinterpret_cast<const PassDesc *>(db + r.desc_off),
                             reinterpret_cast<const uint32_t *>(db + r.tb_off), r.ndesc, r.tiles,
                             ctx->d_err, d_sched + r.sched_idx, r.cost_free, r.fused, ctx->stream);
            break;
        case LK_EIG_INIT:
            e = launch_eig_init(r.iX, r.iX_lo, r.ick0, r.ep.M, r.ep.ld, r.ep.nsets, r.ep.cost, r.ep.cost_dtype,
                                r.ep.coef, r.ep.coef_stride, r.iinit, r.iamp0, ctx->stream);
            break;
        case LK_EIG_GEMM:
            if (r.grouped)
                e = r.tc ? launch_eig_gemm_tc_grouped(r.tm[0], r.tm[1], r.tm[2], r.tm[3], r.Np, r.gtiles, r.n_mtiles,
                                                      r.ep, ctx->d_err, ctx->stream)
                         : launch_eig_gemm_simt_grouped(r.gA, r.lda, r.gB, r.ldb, r.Np, r.gtiles, r.n_mtiles, r.ep,
                                                        ctx->stream);
            else
                e = r.tc ? launch_eig_gemm_tc(r.tm[0], r.tm[1], r.tm[2], r.tm[3], r.Mp, r.Np, r.Kp, r.ep, d_split_ws,
                                              d_split_cnt, ctx->d_err, ctx->stream)
                         : launch_eig_gemm_simt(r.gA, r.gB, r.Mp, r.Np, r.Kp, r.ep, ctx->stream);
            break;
        case LK_ORBIT:
            e = launch_orbit(r.otab, r.oarg, ctx->stream);
            break;
        case LK_OPERANDS:
            e = enqueue_operands(r, ctx->stream);
            break;
        case LK_R1_PASS:
            e = launch_r1_pass(r.r1mode, r.cost_dtype, reinterpret_cast<const R1Desc *>(db + r.desc_off),
                               reinterpret_cast<const uint32_t *>(db + r.tb_off), r.ndesc, r.tiles, r.r1grid,
                               r.r1round, ctx->d_err, ctx->stream);
            break;
        case LK_R1_SCALAR:
            e = launch_r1_scalar(r.r1mode, reinterpret_cast<const R1Desc *>(db + r.desc_off),
                                 reinterpret_cast<const uint32_t *>(db + r.tb_off), r.ndesc, r.r1grid, r.r1round,
                                 ctx->stream);
            break;
        case LK_COST_MEAN:
            e = launch_cost_mean(r.ep.cost, r.ep.cost_dtype, r.ep.M, r.mean_out, ctx->stream);
            break;
        case LK_REDUCE:
            e = launch_reduce(reinterpret_cast<const RedChunk *>(db + r.desc_off), r.ndesc,
                              static_cast<double *>(ctx->bufs["level2"].p),
                              reinterpret_cast<const RedOut *>(db + r.tb_off), (int)r.tiles, ctx->stream);
            break;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
        ctx->launches++;
        if (prof) {
            cudaEventRecord(eb, ctx->stream);
            ctx->pending.push_back({r.fam, ea, eb});
            ctx->fam_stats[r.fam].launches++;
            ctx->fam_stats[r.fam].bytes += r.bytes;
            ctx->fam_stats[r.fam].flops += r.flops;
        }
    }
    return QAOA_OK;
}

qaoa_status check_args(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, const qaoa_mixer *mx,
                         const void *d_init, int p) {
    if (!ctx) return QAOA_ERR_INVALID;
    if (!mx) return fail(ctx, QAOA_ERR_INVALID, "mixer is NULL");
    if (mx->kind == QAOA_MIXER_EIGEN || mx->kind == QAOA_MIXER_EIGEN_SYM) {
        if (!mx->d_V || !mx->d_lambda || ((uintptr_t)mx->d_V & 15) || ((uintptr_t)mx->d_lambda & 7))
            return fail(ctx, QAOA_ERR_INVALID, "eigenbasis mixer needs aligned d_V and d_lambda");
        if (mx->dim < 1 || mx->dim > kMaxEigDim)
            return fail(ctx, QAOA_ERR_INVALID, "eigenbasis mixer dim must be in [1, %d]", kMaxEigDim);
        if (mx->kind == QAOA_MIXER_EIGEN_SYM) {
            if (mx->n < 2 || mx->n > kSymMaxN || mx->k < 0 || mx->k > mx->n)
                return fail(ctx, QAOA_ERR_INVALID, "block XY mixer needs 2 <= n <= %d and 0 <= k <= n", kSymMaxN);
            double D = 1.0;
            for (int i = 0; i < mx->k; i++) D = D * (mx->n - i) / (i + 1);
            if ((int64_t)std::llround(D) != mx->dim)
                return fail(ctx, QAOA_ERR_INVALID, "block XY mixer: dim %lld is not C(%d, %d)", (long long)mx->dim,
                            mx->n, mx->k);
        }
        if (mx->gemm_precision < QAOA_GEMM_FP32_SIMT || mx->gemm_precision > QAOA_GEMM_BF16X3)
            return fail(ctx, QAOA_ERR_INVALID, "unknown GEMM precision %d", mx->gemm_precision);
        if (p < 1 || p > 4096) return fail(ctx, QAOA_ERR_INVALID, "p must be in [1, 4096] (got %d)", p);
        if (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8)
            return fail(ctx, QAOA_ERR_INVALID, "unknown cost dtype %d", cost_dtype);
        if (!d_cost || ((uintptr_t)d_cost & 15))
            return fail(ctx, QAOA_ERR_INVALID, "d_cost must be a 16-byte aligned device pointer");
        if (d_init && ((uintptr_t)d_init & 7)) return fail(ctx, QAOA_ERR_INVALID, "d_init must be 8-byte aligned");
        return QAOA_OK;
    }
    if (mx->kind == QAOA_MIXER_GROVER) {
        if (mx->dim < 1 || mx->dim > kMaxGroverDim)
            return fail(ctx, QAOA_ERR_INVALID, "Grover mixer dim must be in [1, 2^36] (got %lld)", (long long)mx->dim);
        if (p < 1 || p > 4096) return fail(ctx, QAOA_ERR_INVALID, "p must be in [1, 4096] (got %d)", p);
        if (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8)
            return fail(ctx, QAOA_ERR_INVALID, "unknown cost dtype %d", cost_dtype);
        if (!d_cost || ((uintptr_t)d_cost & 15))
            return fail(ctx, QAOA_ERR_INVALID, "d_cost must be a 16-byte aligned device pointer");
        if (d_init && ((uintptr_t)d_init & 15))
            return fail(ctx, QAOA_ERR_INVALID, "d_init must be 16-byte aligned");
        return QAOA_OK;
    }
    if (mx->kind != QAOA_MIXER_X && mx->kind != QAOA_MIXER_X_MA && mx->kind != QAOA_MIXER_X_GENERAL)
        return fail(ctx, QAOA_ERR_INVALID, "unknown mixer kind %d", mx->kind);
    if (mx->kind == QAOA_MIXER_X_GENERAL && (!mx->d_lambda || ((uintptr_t)mx->d_lambda & 7)))
        return fail(ctx, QAOA_ERR_INVALID, "general X mixer needs its n + 1 weights in d_lambda");
    if (mx->n < 1 || mx->n > kMaxXQubits)
        return fail(ctx, QAOA_ERR_INVALID, "X mixer needs 1 <= n <= %d (got %d)", kMaxXQubits, mx->n);
    if (mx->dim != (1ll << mx->n))
        return fail(ctx, QAOA_ERR_INVALID, "X mixer dim must be 2^n (n=%d, dim=%lld)", mx->n,
                    (long long)mx->dim);
    if (p < 1 || p > 4096) return fail(ctx, QAOA_ERR_INVALID, "p must be in [1, 4096] (got %d)", p);
    if (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8)
        return fail(ctx, QAOA_ERR_INVALID, "unknown cost dtype %d", cost_dtype);
    if (!d_cost || ((uintptr_t)d_cost & 15))
        return fail(ctx, QAOA_ERR_INVALID, "d_cost must be a 16-byte aligned device pointer");
    if (d_init && ((uintptr_t)d_init & 15))
        return fail(ctx, QAOA_ERR_INVALID, "d_init must be 16-byte aligned");
    return QAOA_OK;
}

qaoa_status read_dev_err(qaoa_ctx *ctx) {
    int h = 0;
    QG_CUDA(ctx, cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
            "error word read");
    QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
    if (h) {
        cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream);
        if (h & DERR_BAD_ANGLE) return fail(ctx, QAOA_ERR_INVALID, "non-finite angle");
        if (h & DERR_TIMEOUT) return fail(ctx, QAOA_ERR_TIMEOUT, "a bounded device-side wait gave up");
        return fail(ctx, QAOA_ERR_CUDA, "device error word 0x%x", h);
    }
    return QAOA_OK;
}

qaoa_status scalar_run(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, const qaoa_mixer *mixer,
                       const void *d_init, int p, const double *angles, double *E, double *grad,
                       int ckpt) {
    qaoa_status st = check_args(ctx, d_cost, cost_dtype, mixer, d_init, p);
    if (st) return st;
    if (!angles || !E || (grad == nullptr) != (ckpt < 0))
        return fail(ctx, QAOA_ERR_INVALID, "angles and result pointers must be non-NULL");
    const int ma = mixer->kind == QAOA_MIXER_X_MA;
    const int na = ma ? p * (mixer->n + 1) : 2 * p;  // angles (and partials) per set
    for (int i = 0; i < na; i++)
        if (!std::isfinite(angles[i])) return fail(ctx, QAOA_ERR_INVALID, "angle %d is not finite", i);
    const size_t cnt = (size_t)2 * na + 1;
    void *d_io = nullptr;
    st = scratch(ctx, "io", cnt * sizeof(double), &d_io);
    if (st) return st;
    if (ctx->h_io_count < cnt) {
        if (ctx->h_io) {
            cudaStreamSynchronize(ctx->stream);
            cudaFreeHost(ctx->h_io);
        }
        ctx->h_io = nullptr;
        ctx->h_io_count = 0;
        QG_CUDA(ctx, cudaMallocHost(reinterpret_cast<void **>(&ctx->h_io), cnt * sizeof(double)),
                "cudaMallocHost");
        ctx->h_io_count = cnt;
    }
    std::memcpy(ctx->h_io, angles, sizeof(double) * na);
    double *io = static_cast<double *>(d_io);
    QG_CUDA(ctx, cudaMemcpyAsync(io, ctx->h_io, sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream),
            "angle upload");
    Unit u;
    std::memset(&u, 0, sizeof(u));
    u.cost = d_cost;
    u.cost_dtype = cost_dtype;
    u.n = mixer->n;
    u.p = p;
    u.angles = io;
    u.E = io + na;
    u.grad = grad ? io + na + 1 : nullptr;
    u.init = static_cast<const float2 *>(d_init);
    u.tsize = kPhaseTable;
    u.mixer_kind = (ma || mixer->kind == QAOA_MIXER_X_GENERAL) ? QAOA_MIXER_X : mixer->kind;
    u.ma = ma;
    u.gm = mixer->kind == QAOA_MIXER_X_GENERAL;
    u.wts = u.gm ? mixer->d_lambda : nullptr;
    u.dim = mixer->dim;
    u.V = mixer->d_V;
    u.lam = mixer->d_lambda;
    u.gemm_precision = mixer->gemm_precision;
    u.k = mixer->k;
    u.mixer_id = mixer->id;
    std::vector<Unit> us(1, u);
    st = run_units(ctx, us, grad != nullptr, grad ? ckpt : 0);
    if (st) return st;
    const size_t nout = grad ? (size_t)na + 1 : 1;
    QG_CUDA(ctx, cudaMemcpyAsync(ctx->h_io + na, io + na, sizeof(double) * nout, cudaMemcpyDeviceToHost,
                                 ctx->stream),
            "result download");
    st = read_dev_err(ctx);
    if (st) return st;
    *E = ctx->h_io[na];
    if (grad) std::memcpy(grad, ctx->h_io + na + 1, sizeof(double) * na);
    return QAOA_OK;
}

}  // namespace

// ======================================================================
extern "C" {

qaoa_status qaoa_create(qaoa_ctx **out, int device, void *cuda_stream) {
    if (!out) return QAOA_ERR_INVALID;
    *out = nullptr;
    qaoa_ctx *ctx = nullptr;
    try {
        ctx = new qaoa_ctx();
    } catch (...) {
        return QAOA_ERR_OOM;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete ctx;
        return QAOA_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return QAOA_ERR_CUDA;
    }
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess || upload_binom_table() != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return QAOA_ERR_CUDA;
    }
    *out = ctx;
    return QAOA_OK;
}

void qaoa_destroy(qaoa_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto &pe : ctx->pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_io) cudaFreeHost(ctx->h_io);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
}

const char *qaoa_last_error(const qaoa_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t qaoa_scratch_bytes(const qaoa_ctx *ctx) {
    if (!ctx) return -1;
    int64_t t = 0;
    for (auto &kv : ctx->bufs) t += (int64_t)kv.second.bytes;
    return t;
}

qaoa_status qaoa_cost_precompute(qaoa_ctx *ctx, const qaoa_problem *prob, void *d_cost, int cost_dtype,
                                 int64_t dim) {
    NvtxRange nvtx_range("qaoa_cost_precompute");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (!prob || !d_cost) return fail(ctx, QAOA_ERR_INVALID, "problem and d_cost must be non-NULL");
        const int n = prob->n;
        if (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8)
            return fail(ctx, QAOA_ERR_INVALID, "unknown cost dtype %d", cost_dtype);
        const bool dks = prob->kind == QAOA_PROBLEM_DKS || prob->kind == QAOA_PROBLEM_KVC;
        if (n < 1 || n > (dks ? binom_table_max() : 34))
            return fail(ctx, QAOA_ERR_INVALID, "n=%d out of range", n);
        int64_t want;
        if (dks) {
            if (prob->k < 0 || prob->k > n) return fail(ctx, QAOA_ERR_INVALID, "bad k=%d", prob->k);
            double b = 1;
            for (int i = 0; i < prob->k; i++) b = b * (n - i) / (i + 1);
            want = (int64_t)std::llround(b);
        } else {
            want = 1ll << n;
        }
        if (dim != want)
            return fail(ctx, QAOA_ERR_INVALID, "dim=%lld but the feasible set has %lld states",
                        (long long)dim, (long long)want);
        cudaSetDevice(ctx->device);
        if (prob->kind == QAOA_PROBLEM_MAXCUT || prob->kind == QAOA_PROBLEM_WMAXCUT || dks) {
            if (prob->m < 0 || (prob->m > 0 && !prob->edges))
                return fail(ctx, QAOA_ERR_INVALID, "edge list missing");
            uint64_t nbr[64] = {0};
            for (int e = 0; e < prob->m; e++) {
                int u = prob->edges[2 * e], v = prob->edges[2 * e + 1];
                if (u < 0 || v < 0 || u >= n || v >= n || u == v)
                    return fail(ctx, QAOA_ERR_INVALID, "edge %d = (%d,%d) invalid for n=%d", e, u, v, n);
                if (u > v) std::swap(u, v);
                if (nbr[u] & (1ull << v))
                    return fail(ctx, QAOA_ERR_INVALID, "edge (%d,%d) repeated", u, v);
                nbr[u] |= 1ull << v;
            }
            if (cost_dtype == QAOA_COST_U8 && prob->m > 255 && prob->kind != QAOA_PROBLEM_WMAXCUT)
                return fail(ctx, QAOA_ERR_INVALID, "%d edges: costs may exceed 255, use float32", prob->m);
            cudaError_t e;
            if (prob->kind == QAOA_PROBLEM_WMAXCUT) {
                if (cost_dtype != QAOA_COST_F32 || !prob->weights)
                    return fail(ctx, QAOA_ERR_INVALID, "weighted MaxCut needs weights and float32 costs");
                void *dw = nullptr, *de = nullptr;
                qaoa_status st = scratch(ctx, "pre_w", sizeof(float) * std::max(1, prob->m), &dw);
                if (st) return st;
                st = scratch(ctx, "pre_e", sizeof(int32_t) * 2 * std::max(1, prob->m), &de);
                if (st) return st;
                QG_CUDA(ctx, cudaMemcpyAsync(dw, prob->weights, sizeof(float) * prob->m, cudaMemcpyHostToDevice,
                                             ctx->stream), "weights upload");
                QG_CUDA(ctx, cudaMemcpyAsync(de, prob->edges, sizeof(int32_t) * 2 * prob->m,
                                             cudaMemcpyHostToDevice, ctx->stream), "edges upload");
                e = launch_cost_maxcut(n, nbr, static_cast<float *>(dw), static_cast<int32_t *>(de), prob->m, 1,
                                       dim, d_cost, cost_dtype, ctx->stream);
            } else if (dks) {
                e = launch_cost_dks(n, prob->k, nbr, dim, d_cost, cost_dtype, prob->kind == QAOA_PROBLEM_KVC ? 1 : 0,
                                    prob->m, ctx->stream);
            } else {
                e = launch_cost_maxcut(n, nbr, nullptr, nullptr, prob->m, 0, dim, d_cost, cost_dtype,
                                       ctx->stream);
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cost kernel launch");
            ctx->launches++;
        } else if (prob->kind == QAOA_PROBLEM_SK) {
            if (!prob->J) return fail(ctx, QAOA_ERR_INVALID, "SK needs J");
            if (cost_dtype != QAOA_COST_F32) return fail(ctx, QAOA_ERR_INVALID, "SK costs are float32");
            if (n > 40) return fail(ctx, QAOA_ERR_INVALID, "SK supports n <= 40");
            bool exact = true;
            std::vector<int32_t> Jq(n * n, 0);
            std::vector<double> Jd(n * n, 0.0);
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    const double v = (double)prob->J[i * n + j];
                    if (!std::isfinite(v)) return fail(ctx, QAOA_ERR_INVALID, "J[%d][%d] not finite", i, j);
                    Jd[i * n + j] = v;
                    const double q = v * 1048576.0;
                    if (std::fabs(v) >= 8.0 || q != std::rint(q)) exact = false;
                    else Jq[i * n + j] = (int32_t)q;
                }
            void *dj = nullptr;
            qaoa_status st = scratch(ctx, "pre_J", sizeof(double) * n * n, &dj);
            if (st) return st;
            cudaError_t e;
            if (exact) {
                QG_CUDA(ctx, cudaMemcpyAsync(dj, Jq.data(), sizeof(int32_t) * n * n, cudaMemcpyHostToDevice,
                                             ctx->stream), "J upload");
                e = launch_cost_sk(n, static_cast<int32_t *>(dj), nullptr, 1, dim, static_cast<float *>(d_cost),
                                   ctx->stream);
            } else {
                QG_CUDA(ctx, cudaMemcpyAsync(dj, Jd.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice,
                                             ctx->stream), "J upload");
                e = launch_cost_sk(n, nullptr, static_cast<double *>(dj), 0, dim, static_cast<float *>(d_cost),
                                   ctx->stream);
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cost kernel launch");
            ctx->launches++;
        } else {
            return fail(ctx, QAOA_ERR_INVALID, "unknown problem kind %d", prob->kind);
        }
        QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "cost precompute");
        return QAOA_OK;
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_dicke_states(qaoa_ctx *ctx, int n, int k, uint64_t *d_states, int64_t dim) {
    NvtxRange nvtx_range("qaoa_dicke_states");
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->err.clear();
    if (n < 1 || n > binom_table_max() || k < 0 || k > n || !d_states)
        return fail(ctx, QAOA_ERR_INVALID, "bad Dicke arguments n=%d k=%d", n, k);
    double b = 1;
    for (int i = 0; i < k; i++) b = b * (n - i) / (i + 1);
    if (dim != (int64_t)std::llround(b)) return fail(ctx, QAOA_ERR_INVALID, "dim must be binom(n,k)");
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_dicke_states(n, k, dim, d_states, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dicke kernel launch");
    ctx->launches++;
    QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "dicke states");
    return QAOA_OK;
}

qaoa_status qaoa_ring_hamiltonian(qaoa_ctx *ctx, int n, int k, double *d_H, int64_t dim) {
    NvtxRange nvtx_range("qaoa_ring_hamiltonian");
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->err.clear();
    if (n < 3 || n > binom_table_max() || k < 0 || k > n || !d_H)
        return fail(ctx, QAOA_ERR_INVALID, "ring mixer needs 3 <= n <= %d and 0 <= k <= n",
                    binom_table_max());
    double b = 1;
    for (int i = 0; i < k; i++) b = b * (n - i) / (i + 1);
    if (dim != (int64_t)std::llround(b)) return fail(ctx, QAOA_ERR_INVALID, "dim must be binom(n,k)");
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_ring_hamiltonian(n, k, dim, d_H, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ring kernel launch");
    ctx->launches++;
    QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "ring hamiltonian");
    return QAOA_OK;
}

qaoa_status qaoa_clique_hamiltonian(qaoa_ctx *ctx, int n, int k, double *d_H, int64_t dim) {
    NvtxRange nvtx_range("qaoa_clique_hamiltonian");
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->err.clear();
    if (n < 2 || n > binom_table_max() || k < 0 || k > n || !d_H)
        return fail(ctx, QAOA_ERR_INVALID, "clique mixer needs 2 <= n <= %d and 0 <= k <= n",
                    binom_table_max());
    double b = 1;
    for (int i = 0; i < k; i++) b = b * (n - i) / (i + 1);
    if (dim != (int64_t)std::llround(b)) return fail(ctx, QAOA_ERR_INVALID, "dim must be binom(n,k)");
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_clique_hamiltonian(n, k, dim, d_H, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clique kernel launch");
    ctx->launches++;
    QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "clique hamiltonian");
    return QAOA_OK;
}

qaoa_status qaoa_expectation(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, const qaoa_mixer *mixer,
                             const void *d_init, int p, const double *angles, double *E) {
    NvtxRange nvtx_range("qaoa_expectation");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        cudaSetDevice(ctx->device);
        return scalar_run(ctx, d_cost, cost_dtype, mixer, d_init, p, angles, E, nullptr, -1);
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_gradient(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, const qaoa_mixer *mixer,
                          const void *d_init, int p, const double *angles, double *E, double *grad,
                          int ckpt) {
    NvtxRange nvtx_range("qaoa_gradient");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (!grad) return fail(ctx, QAOA_ERR_INVALID, "grad must be non-NULL");
        if (ckpt < QAOA_CKPT_NONE || ckpt > QAOA_CKPT_PASS)
            return fail(ctx, QAOA_ERR_INVALID, "ckpt must be one of QAOA_CKPT_NONE/ROUND/PASS (got %d)", ckpt);
        cudaSetDevice(ctx->device);
        return scalar_run(ctx, d_cost, cost_dtype, mixer, d_init, p, angles, E, grad, ckpt);
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_expectation_batched(qaoa_ctx *ctx, int n_jobs, const qaoa_job *jobs, int want_grad) {
    NvtxRange nvtx_range("qaoa_expectation_batched");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (n_jobs < 1 || !jobs) return fail(ctx, QAOA_ERR_INVALID, "no jobs");
        cudaSetDevice(ctx->device);
        std::vector<Unit> units;
        for (int j = 0; j < n_jobs; j++) {
            const qaoa_job &jb = jobs[j];
            qaoa_status st = check_args(ctx, jb.d_cost, jb.cost_dtype, jb.mixer, jb.d_init, jb.p);
            if (st) return st;
            if (jb.n_sets < 1 || !jb.d_angles || !jb.d_E || (want_grad && !jb.d_grad))
                return fail(ctx, QAOA_ERR_INVALID, "job %d: bad sets or output pointers", j);
            const int ma = jb.mixer->kind == QAOA_MIXER_X_MA;
            const int64_t na = ma ? (int64_t)jb.p * (jb.mixer->n + 1) : 2 * (int64_t)jb.p;
            for (int s = 0; s < jb.n_sets; s++) {
                Unit u;
                std::memset(&u, 0, sizeof(u));
                u.cost = jb.d_cost;
                u.cost_dtype = jb.cost_dtype;
                u.n = jb.mixer->n;
                u.p = jb.p;
                u.angles = jb.d_angles + (int64_t)s * na;
                u.E = jb.d_E + s;
                u.grad = want_grad ? jb.d_grad + (int64_t)s * na : nullptr;
                u.init = static_cast<const float2 *>(jb.d_init);
                u.tsize = kPhaseTable;
                u.mixer_kind = (ma || jb.mixer->kind == QAOA_MIXER_X_GENERAL) ? QAOA_MIXER_X : jb.mixer->kind;
                u.ma = ma;
                u.gm = jb.mixer->kind == QAOA_MIXER_X_GENERAL;
                u.wts = u.gm ? jb.mixer->d_lambda : nullptr;
                u.job = j;
                u.dim = jb.mixer->dim;
                u.V = jb.mixer->d_V;
                u.lam = jb.mixer->d_lambda;
                u.gemm_precision = jb.mixer->gemm_precision;
                u.k = jb.mixer->k;
                u.mixer_id = jb.mixer->id;
                units.push_back(u);
            }
        }
        return run_units(ctx, units, want_grad != 0, want_grad ? ctx->ckpt_mode : 0);
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_expectation_batched_host(qaoa_ctx *ctx, int n_jobs, const qaoa_host_job *jobs, int want_grad) {
    NvtxRange nvtx_range("qaoa_expectation_batched_host");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (n_jobs < 1 || !jobs) return fail(ctx, QAOA_ERR_INVALID, "no jobs");
        if (capturing(ctx)) return fail(ctx, QAOA_ERR_INVALID, "the host-buffer call synchronises; do not capture it");
        cudaSetDevice(ctx->device);
        // device staging, job after job: angles, <C>, gradients
        std::vector<int64_t> na(n_jobs);
        size_t total = 0;
        for (int j = 0; j < n_jobs; j++) {
            const qaoa_host_job &jb = jobs[j];
            if (!jb.mixer) return fail(ctx, QAOA_ERR_INVALID, "job %d: mixer is NULL", j);
            if (jb.p < 1 || jb.p > 4096) return fail(ctx, QAOA_ERR_INVALID, "job %d: p must be in [1, 4096]", j);
            if (jb.n_sets < 1 || !jb.h_angles || !jb.h_E || (want_grad && !jb.h_grad))
                return fail(ctx, QAOA_ERR_INVALID, "job %d: bad sets or host pointers", j);
            na[j] = jb.mixer->kind == QAOA_MIXER_X_MA ? (int64_t)jb.p * (jb.mixer->n + 1) : 2 * (int64_t)jb.p;
            total += (size_t)jb.n_sets * (size_t)(na[j] * (want_grad ? 2 : 1) + 1);
        }
        void *stage = nullptr;
        qaoa_status st = scratch(ctx, "host_io", total * sizeof(double), &stage);
        if (st) return st;
        std::vector<qaoa_job> dj(n_jobs);
        double *cur = static_cast<double *>(stage);
        for (int j = 0; j < n_jobs; j++) {
            const qaoa_host_job &jb = jobs[j];
            const int64_t ns = jb.n_sets, a = ns * na[j];
            qaoa_job &d = dj[j];
            d.d_cost = jb.d_cost;
            d.cost_dtype = jb.cost_dtype;
            d.mixer = jb.mixer;
            d.p = jb.p;
            d.n_sets = jb.n_sets;
            d.d_angles = cur;
            d.d_E = cur + a;
            d.d_grad = want_grad ? cur + a + ns : nullptr;
            d.d_init = jb.d_init;
            QG_CUDA(ctx, cudaMemcpyAsync(cur, jb.h_angles, (size_t)a * sizeof(double), cudaMemcpyHostToDevice,
                                         ctx->stream),
                    "angle upload");
            cur += a + ns + (want_grad ? a : 0);
        }
        st = qaoa_expectation_batched(ctx, n_jobs, dj.data(), want_grad);
        if (st) {
            cudaStreamSynchronize(ctx->stream);  // the uploads read the caller's buffers
            return st;
        }
        for (int j = 0; j < n_jobs; j++) {
            const qaoa_host_job &jb = jobs[j];
            QG_CUDA(ctx, cudaMemcpyAsync(jb.h_E, dj[j].d_E, (size_t)jb.n_sets * sizeof(double),
                                         cudaMemcpyDeviceToHost, ctx->stream),
                    "result download");
            if (want_grad)
                QG_CUDA(ctx, cudaMemcpyAsync(jb.h_grad, dj[j].d_grad, (size_t)jb.n_sets * na[j] * sizeof(double),
                                             cudaMemcpyDeviceToHost, ctx->stream),
                        "gradient download");
        }
        return read_dev_err(ctx);  // synchronises the stream
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_cost_degeneracy(qaoa_ctx *ctx, const qaoa_problem *prob, int64_t *d_counts, int n_bins) {
    NvtxRange nvtx_range("qaoa_cost_degeneracy");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (!prob || !d_counts) return fail(ctx, QAOA_ERR_INVALID, "problem and d_counts must be non-NULL");
        const int n = prob->n, k = prob->k, m = prob->m;
        const bool weighted_k = prob->kind == QAOA_PROBLEM_DKS || prob->kind == QAOA_PROBLEM_KVC;
        if (!weighted_k && !(prob->kind == QAOA_PROBLEM_MAXCUT && k < 0))
            return fail(ctx, QAOA_ERR_UNSUPPORTED, "degeneracies are counted for MAXCUT (k = -1), DKS and KVC");
        if (n < 1 || n > (weighted_k ? 128 : 44))
            return fail(ctx, QAOA_ERR_INVALID, "n=%d out of range (MAXCUT <= 44, DKS/KVC <= 128)", n);
        if (weighted_k && (k < 0 || k > n)) return fail(ctx, QAOA_ERR_INVALID, "bad k=%d", k);
        if (m < 0 || (m > 0 && !prob->edges)) return fail(ctx, QAOA_ERR_INVALID, "edge list missing");
        // the largest cost the problem can take: m edges, at most C(k, 2)
        // inside a k-subset
        int maxc = m;
        if (prob->kind == QAOA_PROBLEM_DKS) maxc = std::min<int64_t>(m, (int64_t)k * (k - 1) / 2);
        if (n_bins <= maxc || n_bins > grover_max_bins())
            return fail(ctx, QAOA_ERR_INVALID, "n_bins=%d must exceed the largest possible cost %d and be <= %d",
                        n_bins, maxc, grover_max_bins());
        // feasible-set size, exactly, with a cap on the enumeration
        const uint64_t kCap = 1ull << 44;
        uint64_t N = 1;
        if (weighted_k) {
            const int kk = std::min(k, n - k);
            long double b = 1;
            for (int i = 0; i < kk; i++) b = b * (n - i) / (i + 1);
            if (b > (long double)kCap) return fail(ctx, QAOA_ERR_UNSUPPORTED, "C(%d,%d) > 2^44 states", n, k);
            N = (uint64_t)std::llround((double)b);
        } else {
            N = 1ull << n;
        }
        DegLaunch L;
        std::memset(&L, 0, sizeof(L));
        for (int e = 0; e < m; e++) {
            int u = prob->edges[2 * e], v = prob->edges[2 * e + 1];
            if (u < 0 || v < 0 || u >= n || v >= n || u == v)
                return fail(ctx, QAOA_ERR_INVALID, "edge %d = (%d,%d) invalid for n=%d", e, u, v, n);
            if (u > v) std::swap(u, v);
            uint64_t &w = v < 64 ? L.up_lo[u] : L.up_hi[u];
            const uint64_t bitv = 1ull << (v & 63);
            if (w & bitv) return fail(ctx, QAOA_ERR_INVALID, "edge (%d,%d) repeated", u, v);
            w |= bitv;
            (u < 64 ? L.up_lo[v] : L.up_hi[v]) |= 1ull << (u & 63);  // both directions
            if (!weighted_k) {
                L.adj[u] |= 1ull << v;
                L.adj[v] |= 1ull << u;
                L.deg[u]++;
                L.deg[v]++;
            }
        }
        L.n = n;
        L.k = k;
        L.m = m;
        L.kind = prob->kind == QAOA_PROBLEM_MAXCUT ? 0 : (prob->kind == QAOA_PROBLEM_DKS ? 1 : 2);
        L.comp = weighted_k && 2 * k > n ? 1 : 0;
        L.n_bins = n_bins;
        cudaSetDevice(ctx->device);
        // binomial coefficients C(a, b), a, b <= 128, saturating at 2^64 - 1
        void *d_binom = nullptr;
        const bool fresh = !ctx->bufs.count("binom128");
        qaoa_status st = scratch(ctx, "binom128", sizeof(uint64_t) * 129 * 129, &d_binom);
        if (st) return st;
        if (fresh) {
            std::vector<uint64_t> h(129 * 129, 0);
            for (int a = 0; a <= 128; a++)
                for (int b = 0; b <= 128; b++) {
                    uint64_t v;
                    if (b == 0) v = 1;
                    else if (a == 0) v = 0;
                    else {
                        const uint64_t x = h[(a - 1) * 129 + b - 1], y = h[(a - 1) * 129 + b];
                        v = (x > ~0ull - y) ? ~0ull : x + y;
                    }
                    h[a * 129 + b] = v;
                }
            QG_CUDA(ctx, cudaMemcpyAsync(d_binom, h.data(), sizeof(uint64_t) * h.size(), cudaMemcpyHostToDevice,
                                         ctx->stream),
                    "binomial table upload");
            QG_CUDA(ctx, cudaStreamSynchronize(ctx->stream), "binomial table upload");
        }
        QG_CUDA(ctx, cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * n_bins, ctx->stream), "counts clear");
        if (const int kk = degeneracy_sliced_kk(L)) {
            // bit-sliced count: all (kk-1)-sets T, each with the v < min(T)
            uint64_t NT = 1;
            for (int i = 0; i < kk - 1; i++) NT = NT * (uint64_t)(n - i) / (uint64_t)(i + 1);
            // each T adds at most 127 to one thread's 32-bit counter per value
            const uint64_t tslab = 1ull << 34;
            for (uint64_t t0 = 0; t0 < NT; t0 += tslab) {
                cudaError_t e = launch_degeneracy_sliced(L, static_cast<const uint64_t *>(d_binom), t0,
                                                         std::min(tslab, NT - t0),
                                                         reinterpret_cast<unsigned long long *>(d_counts),
                                                         ctx->d_err, ctx->stream);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "degeneracy kernel launch");
                ctx->launches++;
            }
            return read_dev_err(ctx);
        }
        const uint64_t slab = 1ull << 36;  // keeps every warp's 32-bit shared counters from wrapping
        for (uint64_t s0 = 0; s0 < N; s0 += slab) {
            const uint64_t cnt = std::min(slab, N - s0);
            cudaError_t e = launch_degeneracy(L, static_cast<const uint64_t *>(d_binom), s0, cnt,
                                              reinterpret_cast<unsigned long long *>(d_counts), ctx->d_err,
                                              ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "degeneracy kernel launch");
            ctx->launches++;
        }
        return read_dev_err(ctx);
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_grover_batched(qaoa_ctx *ctx, const int64_t *d_counts, int n_bins, int p, int n_sets,
                                const double *d_angles, double *d_E, double *d_grad) {
    NvtxRange nvtx_range("qaoa_grover_batched");
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->err.clear();
    if (!d_counts || !d_angles || !d_E) return fail(ctx, QAOA_ERR_INVALID, "counts, angles and E must be non-NULL");
    if (n_bins < 1 || n_bins > grover_max_bins())
        return fail(ctx, QAOA_ERR_INVALID, "n_bins must be in [1, %d]", grover_max_bins());
    if (p < 1 || p > 1024 || n_sets < 1)
        return fail(ctx, QAOA_ERR_INVALID, "p must be in [1, 1024] and n_sets >= 1 (p=%d, n_sets=%d)", p, n_sets);
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_grover_eval(d_counts, n_bins, p, n_sets, d_angles, d_E, d_grad, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "Grover kernel launch");
    ctx->launches++;
    return QAOA_OK;
}

qaoa_status qaoa_check_bounded_wait(qaoa_ctx *ctx) {
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->err.clear();
    cudaSetDevice(ctx->device);
    cudaError_t e = launch_wait_probe(ctx->d_err, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait probe launch");
    ctx->launches++;
    return read_dev_err(ctx);
}

qaoa_status qaoa_set_checkpointing(qaoa_ctx *ctx, int mode) {
    if (!ctx) return QAOA_ERR_INVALID;
    if (mode < QAOA_CKPT_NONE || mode > QAOA_CKPT_PASS)
        return fail(ctx, QAOA_ERR_INVALID, "checkpoint mode must be 0, 1 or 2 (got %d)", mode);
    ctx->ckpt_mode = mode;
    return QAOA_OK;
}

qaoa_status qaoa_x_mixer_weights(int n, int kmax, const double *c, double *d) {
    if (n < 1 || n > 62 || kmax < 0 || kmax > n || !c || !d) return QAOA_ERR_INVALID;
    // binomials of n <= 62 in exact 64-bit integers (largest C(62, 31) < 2^63)
    std::vector<std::vector<int64_t>> B(n + 1, std::vector<int64_t>(n + 1, 0));
    for (int a = 0; a <= n; a++) {
        B[a][0] = 1;
        for (int b = 1; b <= a; b++) B[a][b] = B[a - 1][b - 1] + (b <= a - 1 ? B[a - 1][b] : 0);
    }
    for (int w = 0; w <= n; w++) {
        double acc = 0.0;
        for (int k = 0; k <= kmax; k++) {
            if (c[k] == 0.0) continue;
            // K_k(w): the value of sum_{|S| = k} prod_{i in S} Z_i on a weight-w
            // basis state; its terms alternate, so it is summed exactly in integers
            // (|K_k(w)| <= C(n, k)) before the one rounding to double
            int64_t K = 0;
            for (int j = 0; j <= k && j <= w; j++) {
                if (k - j > n - w) continue;
                const int64_t t = B[w][j] * B[n - w][k - j];
                K += (j & 1) ? -t : t;
            }
            acc += c[k] * (double)K;
        }
        d[w] = acc;
    }
    return QAOA_OK;
}

qaoa_status qaoa_set_state_limit(qaoa_ctx *ctx, int64_t bytes) {
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->state_limit = bytes < 0 ? -1 : bytes;
    ctx->plan.valid = false;  // the next call re-plans its waves under the new cap
    return QAOA_OK;
}

int qaoa_pass_schedule(int n, int cmin, int split, int *c, int *lo, int max) {
    if (n <= kPassTileBits || n > kMaxXQubits || cmin < 4 || cmin > 8 || split < 0 || split > 2) return -1;
    const std::vector<Group> g = make_groups(n, kPassTileBits, cmin, split);
    for (int j = 0; j < (int)g.size() && j < max; j++) {
        if (c) c[j] = g[j].c;
        if (lo) lo[j] = g[j].lo;
    }
    return (int)g.size();
}

qaoa_status qaoa_set_xtune(qaoa_ctx *ctx, const qaoa_xtune *t) {
    if (!ctx || !t) return QAOA_ERR_INVALID;
    if (!valid_xtune(*t))
        return fail(ctx, QAOA_ERR_INVALID,
                    "schedule needs %d < n <= %d, cost dtype 0/1, cmin 4..8, split 0..2, buffers 1 or 2",
                    small_max_n(), kMaxXQubits);
    ctx->xtune[{t->n, t->cost_dtype}] = *t;
    ctx->tune_epoch++;
    return QAOA_OK;
}

qaoa_status qaoa_get_xtune(qaoa_ctx *ctx, int n, int cost_dtype, qaoa_xtune *out) {
    if (!ctx || !out) return QAOA_ERR_INVALID;
    *out = tune_for(ctx, n, cost_dtype);
    return QAOA_OK;
}

qaoa_status qaoa_autotune_x(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, int n, int p, int want_grad,
                            qaoa_xtune *out) {
    NvtxRange nvtx_range("qaoa_autotune_x");
    if (!ctx) return QAOA_ERR_INVALID;
    try {
        ctx->err.clear();
        if (!d_cost || (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8))
            return fail(ctx, QAOA_ERR_INVALID, "bad cost vector or dtype");
        if (n <= small_max_n() || n > kMaxXQubits)
            return fail(ctx, QAOA_ERR_INVALID, "tuning applies to %d < n <= %d (got %d)", small_max_n(),
                        kMaxXQubits, n);
        if (p < 1 || p > 8) return fail(ctx, QAOA_ERR_INVALID, "tuning rounds p must be 1..8 (got %d)", p);
        if (capturing(ctx)) return fail(ctx, QAOA_ERR_INVALID, "cannot tune during stream capture");
        cudaSetDevice(ctx->device);
        // fixed angles (beta away from pi/2, so the rotations take their usual form)
        std::vector<double> h(4 * p + 1, 0.0);
        for (int k = 0; k < p; k++) {
            h[k] = 0.35 + 0.05 * k;
            h[p + k] = 0.25 + 0.03 * k;
        }
        void *d_io = nullptr;
        qaoa_status st = scratch(ctx, "tune_io", h.size() * sizeof(double), &d_io);
        if (st) return st;
        double *io = static_cast<double *>(d_io);
        QG_CUDA(ctx, cudaMemcpyAsync(io, h.data(), sizeof(double) * 2 * p, cudaMemcpyHostToDevice, ctx->stream),
                "tuning angles");
        Unit u;
        std::memset(&u, 0, sizeof(u));
        u.cost = d_cost;
        u.cost_dtype = cost_dtype;
        u.n = n;
        u.p = p;
        u.angles = io;
        u.E = io + 2 * p;
        u.grad = want_grad ? io + 2 * p + 1 : nullptr;
        u.tsize = kPhaseTable;
        u.mixer_kind = QAOA_MIXER_X;
        u.dim = 1ll << n;
        const std::vector<Unit> us(1, u);
        const int ck = want_grad ? ctx->ckpt_mode : 0;
        const bool had = ctx->xtune.count({n, cost_dtype}) != 0;
        const qaoa_xtune saved = tune_for(ctx, n, cost_dtype);
        cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
        auto restore = [&]() {
            if (had) ctx->xtune[{n, cost_dtype}] = saved;
            else ctx->xtune.erase({n, cost_dtype});
            ctx->tune_epoch++;
        };
        // best of three timed sweeps after one untimed sweep that builds the plan
        auto time_it = [&](const qaoa_xtune &t, double *ms) -> qaoa_status {
            ctx->xtune[{n, cost_dtype}] = t;
            ctx->tune_epoch++;
            qaoa_status s2 = run_units(ctx, us, want_grad != 0, ck);
            if (s2) return s2;
            double best = 1e30;
            for (int r = 0; r < 3; r++) {
                cudaEventRecord(e0, ctx->stream);
                s2 = run_units(ctx, us, want_grad != 0, ck);
                if (s2) return s2;
                cudaEventRecord(e1, ctx->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) return read_dev_err(ctx);
                float f = 0.f;
                cudaEventElapsedTime(&f, e0, e1);
                best = std::min(best, (double)f);
            }
            *ms = best;
            return read_dev_err(ctx);
        };
        // 1. pass groups: every (cmin, split) with the fewest passes, distinct
        std::vector<qaoa_xtune> cands;
        std::set<std::vector<int>> seen;
        size_t fewest = 1000;
        for (int cm = 4; cm <= 8; cm++)
            fewest = std::min(fewest, make_groups(n, kPassTileBits, cm, 0).size());
        for (int cm = 4; cm <= 8; cm++) {
            for (int sp = 0; sp <= 2; sp++) {
                const std::vector<Group> g = make_groups(n, kPassTileBits, cm, sp);
                if (g.size() != fewest) continue;
                std::vector<int> sig;
                for (const Group &x : g) {
                    sig.push_back(x.c);
                    sig.push_back(x.lo);
                }
                if (!seen.insert(sig).second) continue;
                qaoa_xtune t = default_xtune(n, cost_dtype);
                t.cmin = cm;
                t.split = sp;
                cands.push_back(t);
            }
        }
        qaoa_xtune best = cands.front();
        best.ms = 1e30;
        for (qaoa_xtune t : cands) {
            double ms = 0.0;
            st = time_it(t, &ms);
            if (st) {
                restore();
                return st;
            }
            if (ms < best.ms) {
                best = t;
                best.ms = ms;
            }
        }
        // 2. adjoint tile buffers, contiguous and gathered passes
        if (want_grad) {
            const qaoa_xtune base = best;
            for (int bc = 1; bc <= 2; bc++) {
                for (int bg = 1; bg <= 2; bg++) {
                    if (bc == base.nbuf_bwd_contig && bg == base.nbuf_bwd_gather) continue;
                    qaoa_xtune t = base;
                    t.nbuf_bwd_contig = bc;
                    t.nbuf_bwd_gather = bg;
                    double ms = 0.0;
                    st = time_it(t, &ms);
                    if (st) {
                        restore();
                        return st;
                    }
                    if (ms < best.ms) {
                        best = t;
                        best.ms = ms;
                    }
                }
            }
        }
        ctx->ev_pool.push_back(e0);
        ctx->ev_pool.push_back(e1);
        ctx->xtune[{n, cost_dtype}] = best;
        ctx->tune_epoch++;
        if (out) *out = best;
        return QAOA_OK;
    } catch (...) {
        return fail(ctx, QAOA_ERR_OOM, "host allocation failed");
    }
}

qaoa_status qaoa_set_profiling(qaoa_ctx *ctx, int enable) {
    if (!ctx) return QAOA_ERR_INVALID;
    ctx->profiling = enable != 0;
    return QAOA_OK;
}

int qaoa_kernel_stats(qaoa_ctx *ctx, qaoa_kernel_stat *out, int max) {
    if (!ctx) return -1;
    cudaSetDevice(ctx->device);
    if (!ctx->pending.empty()) {
        cudaStreamSynchronize(ctx->stream);
        for (auto &pe : ctx->pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) ctx->fam_stats[pe.fam].ms += ms;
            ctx->ev_pool.push_back(pe.a);
            ctx->ev_pool.push_back(pe.b);
        }
        ctx->pending.clear();
    }
    const int nf = (int)ctx->fam_names.size();
    for (int i = 0; i < nf && i < max && out; i++) {
        std::memset(&out[i], 0, sizeof(out[i]));
        std::snprintf(out[i].name, sizeof(out[i].name), "%s", ctx->fam_names[i].c_str());
        out[i].launches = ctx->fam_stats[i].launches;
        out[i].total_ms = ctx->fam_stats[i].ms;
        out[i].algo_bytes = ctx->fam_stats[i].bytes;
        out[i].algo_flops = ctx->fam_stats[i].flops;
    }
    return nf;
}

void qaoa_reset_stats(qaoa_ctx *ctx) {
    if (!ctx) return;
    qaoa_kernel_stats(ctx, nullptr, 0);
    for (auto &s : ctx->fam_stats) s = StatAcc();
    ctx->launches = 0;
}

int64_t qaoa_launch_count(const qaoa_ctx *ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
