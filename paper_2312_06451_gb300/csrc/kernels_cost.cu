// Cost-vector pre-computation over the feasible set (arXiv 2312.06451,
// Sec. 2.1: C(x) is evaluated once for every feasible x and stored) and the
// Hamming-weight-k feasible set itself.
//
//   MaxCut   C(x) = sum_u popcount(nbr_hi[u] & (x_u ? ~x : x)): every edge
//            (u, v), v > u, is counted from its lower end when x_v != x_u.
//   DkS      C(x) = sum_u x_u popcount(nbr_hi[u] & x) on weight-k states.
//   k-VC     C(x) = m - (the DkS count of the complement of x).
//   SK       C(x) = sum_{i<j} J_ij z_i z_j, z_i = 1 - 2 x_i.  When every
//            J_ij is a multiple of 2^-20 the sum is carried exactly in int64
//            (J scaled by 2^20) and rounded once to float32, so the result is
//            independent of summation order.
//   Dicke    state of rank r (increasing integer order = colex order of
//            k-subsets) by the combinatorial number system:
//            x = {c_k > ... > c_1}, r = sum_i binom(c_i, i).
#include "common.cuh"

namespace qg {

constexpr int kBinomMax = 41;  // n <= 40 for weight-k problems
__constant__ uint64_t c_binom[kBinomMax][kBinomMax];

int binom_table_max() { return kBinomMax - 1; }

cudaError_t upload_binom_table() {
    static uint64_t h[kBinomMax][kBinomMax];
    for (int a = 0; a < kBinomMax; a++)
        for (int b = 0; b < kBinomMax; b++)
            h[a][b] = (b == 0) ? 1 : (a == 0 ? 0 : h[a - 1][b - 1] + h[a - 1][b]);
    return cudaMemcpyToSymbol(c_binom, h, sizeof(h));
}

namespace {

struct AdjParams {
    uint64_t nbr[64];
    int n;
};

__device__ __forceinline__ uint64_t unrank_colex(int64_t r, int n, int k) {
    uint64_t x = 0;
    int c = n - 1;
    for (int i = k; i >= 1; i--) {
        while (c_binom[c][i] > (uint64_t)r) c--;
        x |= 1ull << c;
        r -= (int64_t)c_binom[c][i];
        c--;
    }
    return x;
}

__device__ __forceinline__ int64_t rank_colex(uint64_t x) {
    int64_t r = 0;
    int i = 1;
    while (x) {
        const int c = __ffsll((long long)x) - 1;
        r += (int64_t)c_binom[c][i];
        i++;
        x &= x - 1;
    }
    return r;
}

__global__ void cost_maxcut_kernel(AdjParams A, int64_t dim, void *out, int dtype) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < dim;
         x += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        const uint64_t ux = (uint64_t)x;
        for (int u = 0; u < A.n; u++) {
            const uint64_t m = A.nbr[u];
            c += __popcll(m & (((ux >> u) & 1) ? ~ux : ux));
        }
        if (dtype == 1)
            reinterpret_cast<unsigned char *>(out)[x] = (unsigned char)c;
        else
            reinterpret_cast<float *>(out)[x] = (float)c;
    }
}

__global__ void cost_wmaxcut_kernel(const int32_t *edges, const float *w, int m, int64_t dim,
                                    float *out) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < dim;
         x += (int64_t)gridDim.x * blockDim.x) {
        double c = 0.0;
        for (int e = 0; e < m; e++) {
            const int u = __ldg(edges + 2 * e), v = __ldg(edges + 2 * e + 1);
            if (((x >> u) ^ (x >> v)) & 1) c += (double)__ldg(w + e);
        }
        out[x] = (float)c;
    }
}

constexpr int kSkMaxN = 40;

__global__ void cost_sk_exact_kernel(int n, const int32_t *Jq, int64_t dim, float *out) {
    __shared__ int32_t J[kSkMaxN * kSkMaxN];
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) J[i] = Jq[i];
    __syncthreads();
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < dim;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ux = (uint64_t)x;
        int64_t acc = 0;
        for (int i = 0; i < n; i++) {
            const uint64_t xi = (ux >> i) & 1;
            const int32_t *row = J + i * n;
            for (int j = i + 1; j < n; j++) {
                const int32_t v = row[j];
                acc += (((ux >> j) & 1) ^ xi) ? -(int64_t)v : (int64_t)v;
            }
        }
        out[x] = __ll2float_rn(acc) * 9.5367431640625e-07f;  // * 2^-20, exact
    }
}

__global__ void cost_sk_f64_kernel(int n, const double *Jd, int64_t dim, float *out) {
    __shared__ double J[kSkMaxN * kSkMaxN];
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) J[i] = Jd[i];
    __syncthreads();
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < dim;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ux = (uint64_t)x;
        double acc = 0.0;
        for (int i = 0; i < n; i++) {
            const uint64_t xi = (ux >> i) & 1;
            for (int j = i + 1; j < n; j++) {
                const double v = J[i * n + j];
                acc += (((ux >> j) & 1) ^ xi) ? -v : v;
            }
        }
        out[x] = (float)acc;
    }
}

// kvc = 0: edges inside the chosen set (densest k-subgraph); kvc = 1: edges
// with an end in the set (k-vertex cover) = m - edges inside the complement.
__global__ void cost_dks_kernel(AdjParams A, int k, int64_t dim, void *out, int dtype, int kvc, int m) {
    const uint64_t full = A.n == 64 ? ~0ull : ((1ull << A.n) - 1);
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < dim;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x0 = unrank_colex(a, A.n, k);
        const uint64_t x = kvc ? (full ^ x0) : x0;
        int c = 0;
        for (int u = 0; u < A.n; u++)
            if ((x >> u) & 1) c += __popcll(A.nbr[u] & x);
        if (kvc) c = m - c;
        if (dtype == 1)
            reinterpret_cast<unsigned char *>(out)[a] = (unsigned char)c;
        else
            reinterpret_cast<float *>(out)[a] = (float)c;
    }
}

__global__ void dicke_states_kernel(int n, int k, int64_t dim, uint64_t *out) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < dim;
         a += (int64_t)gridDim.x * blockDim.x)
        out[a] = unrank_colex(a, n, k);
}

// Row a of the ring mixer restricted to weight-k states: for every ring edge
// (i, i+1 mod n) whose bits differ, X_i X_j + Y_i Y_j maps |x> to 2|x'> with
// the two bits swapped.  Row a is written only by thread a.
__global__ void ring_h_kernel(int n, int k, int64_t dim, double *H) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < dim;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = unrank_colex(a, n, k);
        for (int i = 0; i < n; i++) {
            const int j = (i + 1) % n;
            if (((x >> i) ^ (x >> j)) & 1) {
                const uint64_t y = x ^ (1ull << i) ^ (1ull << j);
                H[a * dim + rank_colex(y)] += 2.0;
            }
        }
    }
}

// Row a of the clique mixer restricted to weight-k states: the same swap
// term on every pair i < j whose bits differ.
__global__ void clique_h_kernel(int n, int k, int64_t dim, double *H) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < dim;
         a += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = unrank_colex(a, n, k);
        for (int i = 0; i < n; i++) {
            if (!((x >> i) & 1)) continue;  // i: a set bit, j: a clear bit
            for (int j = 0; j < n; j++) {
                if ((x >> j) & 1) continue;
                const uint64_t y = x ^ (1ull << i) ^ (1ull << j);
                H[a * dim + rank_colex(y)] += 2.0;
            }
        }
    }
}

unsigned grid_for(int64_t dim, int threads) {
    int64_t b = (dim + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

AdjParams make_adj(int n, const uint64_t *nbr_hi) {
    AdjParams A;
    for (int i = 0; i < 64; i++) A.nbr[i] = (i < n) ? nbr_hi[i] : 0;
    A.n = n;
    return A;
}

}  // namespace

cudaError_t launch_cost_maxcut(int n, const uint64_t *nbr_hi, const float *d_w, const int32_t *d_edges,
                               int m, int weighted, int64_t dim, void *d_out, int dtype,
                               cudaStream_t s) {
    if (weighted) {
        cost_wmaxcut_kernel<<<grid_for(dim, 256), 256, 0, s>>>(d_edges, d_w, m, dim,
                                                               reinterpret_cast<float *>(d_out));
    } else {
        cost_maxcut_kernel<<<grid_for(dim, 256), 256, 0, s>>>(make_adj(n, nbr_hi), dim, d_out, dtype);
    }
    return cudaGetLastError();
}

cudaError_t launch_cost_sk(int n, const int32_t *d_Jq, const double *d_Jd, int exact, int64_t dim,
                           float *d_out, cudaStream_t s) {
    if (n > kSkMaxN) return cudaErrorInvalidValue;
    if (exact)
        cost_sk_exact_kernel<<<grid_for(dim, 256), 256, 0, s>>>(n, d_Jq, dim, d_out);
    else
        cost_sk_f64_kernel<<<grid_for(dim, 256), 256, 0, s>>>(n, d_Jd, dim, d_out);
    return cudaGetLastError();
}

cudaError_t launch_cost_dks(int n, int k, const uint64_t *nbr_hi, int64_t dim, void *d_out, int dtype,
                            int kvc, int m, cudaStream_t s) {
    cost_dks_kernel<<<grid_for(dim, 256), 256, 0, s>>>(make_adj(n, nbr_hi), k, dim, d_out, dtype, kvc, m);
    return cudaGetLastError();
}

cudaError_t launch_dicke_states(int n, int k, int64_t dim, uint64_t *d_out, cudaStream_t s) {
    dicke_states_kernel<<<grid_for(dim, 256), 256, 0, s>>>(n, k, dim, d_out);
    return cudaGetLastError();
}

cudaError_t launch_ring_hamiltonian(int n, int k, int64_t dim, double *d_H, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_H, 0, (size_t)dim * (size_t)dim * sizeof(double), s);
    if (e != cudaSuccess) return e;
    ring_h_kernel<<<grid_for(dim, 128), 128, 0, s>>>(n, k, dim, d_H);
    return cudaGetLastError();
}

cudaError_t launch_clique_hamiltonian(int n, int k, int64_t dim, double *d_H, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_H, 0, (size_t)dim * (size_t)dim * sizeof(double), s);
    if (e != cudaSuccess) return e;
    clique_h_kernel<<<grid_for(dim, 128), 128, 0, s>>>(n, k, dim, d_H);
    return cudaGetLastError();
}

}  // namespace qg
