// qaoa_gradient_small_noalloc: the small-n expectation / gradient without any
// device allocation, for callers that cannot call cudaMalloc (for example code
// running under a memory manager that forbids allocations after start-up, or a
// host that owns all device memory itself).  The kernel's scratch -- per-round
// rotation and phase coefficients, the phase tables of uint8 costs, the launch
// descriptors and the device error word -- lives in one file-scope device array
// of fixed size instead of context-owned allocations.
#include "qaoa.h"
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {
constexpr size_t kNoAllocBytesDecl = 256 * 1024;
}  // namespace

// The scratch array (file scope, internal linkage).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytesDecl];

namespace {

// Fixed scratch: 256 KiB, enough for p <= kNoAllocMaxP rounds (coefficients
// 32 B and a 2 KiB phase table per round, plus descriptors).  Every device
// that loads the library holds this array until the process exits.
constexpr size_t kNoAllocBytes = kNoAllocBytesDecl;
constexpr int kNoAllocMaxP = 96;
constexpr size_t kOffErr = 0;
constexpr size_t kOffPrep = 64;
constexpr size_t kOffSmall = 192;
constexpr size_t kOffCoef = 512;
constexpr size_t kOffTable = kOffCoef + sizeof(qg::RoundCoef) * kNoAllocMaxP;
static_assert(kOffTable % 256 == 0, "table offset alignment");
static_assert(kOffTable + sizeof(float2) * qg::kPhaseTable * kNoAllocMaxP <= kNoAllocBytes,
              "scratch too small for kNoAllocMaxP rounds");
static_assert(sizeof(qg::PrepDesc) <= kOffSmall - kOffPrep, "descriptor layout");
static_assert(sizeof(qg::SmallDesc) <= kOffCoef - kOffSmall, "descriptor layout");

std::mutex g_mu;
unsigned char *g_dev_ptr[qg::kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in).  The address is
// kept for the life of the process: after cudaDeviceReset the module is loaded
// again and the array may move, so the entry point must not be used after a
// reset of a device it has already run on.
cudaError_t scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= qg::kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" qaoa_status qaoa_gradient_small_noalloc(const void *d_cost, int cost_dtype, int n, int p,
                                                   const double *d_angles, double *d_E, double *d_grad,
                                                   void *cuda_stream) {
    if (n < 1 || n > qg::small_max_n() || p < 1 || p > kNoAllocMaxP) return QAOA_ERR_INVALID;
    if (cost_dtype != QAOA_COST_F32 && cost_dtype != QAOA_COST_U8) return QAOA_ERR_INVALID;
    if (!d_cost || !d_angles || !d_E || ((uintptr_t)d_cost & 15)) return QAOA_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return QAOA_ERR_CUDA;
    }
    int *d_err = reinterpret_cast<int *>(base + kOffErr);
    qg::RoundCoef *coef = reinterpret_cast<qg::RoundCoef *>(base + kOffCoef);
    float2 *table = cost_dtype == QAOA_COST_U8 ? reinterpret_cast<float2 *>(base + kOffTable) : nullptr;

    // descriptors: copied into the array from this stack frame (a pageable
    // source: the copy has consumed it when cudaMemcpyAsync returns)
    unsigned char host[kOffCoef - kOffPrep];
    std::memset(host, 0, sizeof(host));
    qg::PrepDesc pd;
    std::memset(&pd, 0, sizeof(pd));
    pd.angles = d_angles;
    pd.coef = coef;
    pd.table = table;
    pd.p = p;
    pd.tsize = qg::kPhaseTable;
    qg::SmallDesc sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.cost = d_cost;
    sd.init = nullptr;
    sd.coef = coef;
    sd.table = table;
    sd.E_out = d_E;
    sd.grad_out = d_grad;
    sd.n = n;
    sd.p = p;
    sd.amp0 = (float)(1.0 / std::sqrt(std::ldexp(1.0, n)));
    std::memcpy(host, &pd, sizeof(pd));
    std::memcpy(host + (kOffSmall - kOffPrep), &sd, sizeof(sd));

    int h_err = 0;
    if (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemcpyAsync(base + kOffPrep, host, sizeof(host), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        qg::launch_prep(reinterpret_cast<const qg::PrepDesc *>(base + kOffPrep), 1, d_err, s) != cudaSuccess ||
        qg::launch_small(reinterpret_cast<const qg::SmallDesc *>(base + kOffSmall), 1, cost_dtype,
                         d_grad ? 1 : 0, n, d_err, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QAOA_ERR_CUDA;
    }
    if (h_err & qg::DERR_BAD_ANGLE) return QAOA_ERR_INVALID;
    return h_err ? QAOA_ERR_CUDA : QAOA_OK;
}
