// Grover-mixer QAOA on cost degeneracies (arXiv 2312.06451, Sec. 2.4).
//
// With the Grover mixer H_G = |u><u| (u the uniform superposition over the
// feasible set) and the uniform initial state, every feasible state with the
// same cost value keeps the same amplitude ("fair sampling"), so the QAOA
// only needs the distinct cost values c_j and their degeneracies d_j.  The
// heavy part is counting the degeneracies over 2^n (or C(n, k)) states; the
// simulation then runs on a vector of at most a few thousand values.
//
//   degeneracy kernel  every thread walks a contiguous range of the feasible
//                      states and adds one count per state to a per-warp
//                      shared-memory histogram:
//                      * all 2^n states (MaxCut) in Gray-code order: flipping
//                        qubit i changes the cut by deg_i - 2 cut_i(x), where
//                        cut_i(x) = popcount(adj_i & (x_i ? ~x : x)) counts
//                        the cut edges at i, so a step costs one popcount;
//                      * the weight-k states (densest k-subgraph, k-vertex
//                        cover) in increasing integer order: the range start
//                        by the combinatorial number system, the next state by
//                        Gosper's hack (Sec. 2.4), on 128-bit masks (n <= 128);
//                        k > n/2 enumerates the n-k clear bits instead.  The
//                        states {v} u T, v < min(T), have consecutive ranks:
//                        a thread fixes T and sweeps v with one two-word
//                        popcount per state (counted in packed 8-bit register
//                        fields when the cost depends on |N(v) & T| alone).
//   reduced simulation one CTA per angle set: b_j = sqrt(d_j) a_j evolves as a
//                      QAOA on the values with initial state u_j = sqrt(d_j/N)
//                      and mixer e^{-i beta H_G} = I + (e^{-i beta} - 1) u u^T;
//                      forward, <C> = sum_j c_j |b_j|^2 and the adjoint
//                      recurrences, in float64 (the vector is tiny).
#include "common.cuh"

#include <algorithm>
#include <cstring>

namespace qg {
namespace {

// A set of up to 128 vertices as two 64-bit words (bit i of lo = vertex i,
// bit i of hi = vertex 64 + i).
struct Set2 {
    uint64_t lo, hi;
};

// Next larger set of the same size in increasing integer order (Gosper's
// hack): with u the lowest set bit, v = x + u clears x's lowest block of b
// ones and sets the bit above it; v ^ x is that run of b + 1 ones, and its
// b - 1 = popcount(v ^ x) - 2 extra ones go to the bottom.
__device__ __forceinline__ Set2 gosper_next(Set2 x) {
    uint64_t vlo, vhi;
    if (x.lo) {
        vlo = x.lo + (x.lo & (0ull - x.lo));
        vhi = x.hi + (vlo < x.lo ? 1ull : 0ull);
    } else {
        vlo = 0;
        vhi = x.hi + (x.hi & (0ull - x.hi));
    }
    const int c = __popcll(vlo ^ x.lo) + __popcll(vhi ^ x.hi) - 2;
    const uint64_t mlo = c >= 64 ? ~0ull : ((1ull << c) - 1ull);
    const uint64_t mhi = c > 64 ? ((1ull << (c - 64)) - 1ull) : 0ull;
    return {vlo | mlo, vhi | mhi};
}

// Weight-k subset of rank r in increasing integer (colex) order; binom is the
// (129 x 129) table of binomial coefficients, row = n, column = k.
__device__ Set2 unrank_colex128(uint64_t r, int n, int k, const uint64_t *__restrict__ binom) {
    Set2 x = {0ull, 0ull};
    int c = n - 1;
    for (int i = k; i >= 1; i--) {
        while (binom[c * 129 + i] > r) c--;
        if (c < 64) x.lo |= 1ull << c;
        else x.hi |= 1ull << (c - 64);
        r -= binom[c * 129 + i];
        c--;
    }
    return x;
}

constexpr int kDegThreads = 256;
constexpr int kDegWarps = kDegThreads / 32;

// Count one state of cost c; a cost outside the histogram (which valid
// input never produces) is recorded instead of written.
__device__ __forceinline__ void add_bin(uint32_t *h, int c, int n_bins, bool &bad) {
    if ((unsigned)c < (unsigned)n_bins) atomicAdd(&h[c], 1u);
    else bad = true;
}

struct DegParams {
    uint64_t up_lo[128], up_hi[128];  // all neighbours of u (weight-k problems)
    uint64_t adj[64];                 // all neighbours (MaxCut, n <= 63)
    int deg[64];
    int n, k, m, kind;                // kind: 0 MaxCut, 1 DkS, 2 k-vertex cover
    int comp;                         // weight-k: enumerate the clear bits
};

__global__ void __launch_bounds__(kDegThreads)
degeneracy_kernel(const DegParams P, const uint64_t *__restrict__ binom, uint64_t start, uint64_t count,
                  int n_bins, int copies, unsigned long long *__restrict__ counts, int *err) {
    extern __shared__ uint32_t hist[];  // copies x n_bins
    // adjacency in shared memory: threads index it with different vertices
    __shared__ uint64_t s_up_lo[128], s_up_hi[128], s_adj[64];
    __shared__ int s_deg[64], s_deg2[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        s_up_lo[i] = P.up_lo[i];
        s_up_hi[i] = P.up_hi[i];
        s_deg2[i] = __popcll(P.up_lo[i]) + __popcll(P.up_hi[i]);
        if (i < 64) {
            s_adj[i] = P.adj[i];
            s_deg[i] = P.deg[i];
        }
    }
    for (int i = threadIdx.x; i < copies * n_bins; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    uint32_t *h = hist + (size_t)((threadIdx.x >> 5) % copies) * n_bins;

    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t per = (count + T - 1) / T;
    const uint64_t a0 = start + tid * per;
    const uint64_t a1 = min(start + count, a0 + per);
    if (a0 < a1) {
        if (P.kind == 0) {
            // Gray-code walk: state g(a) = a ^ (a >> 1); from a to a + 1 the
            // qubit ctz(a + 1) flips
            uint64_t x = a0 ^ (a0 >> 1);
            int cut = 0;
            for (int u = 0; u < P.n; u++)
                if ((x >> u) & 1) cut += __popcll(s_adj[u] & ~x);
            bool bad = false;
            add_bin(h, cut, n_bins, bad);
            for (uint64_t a = a0 + 1; a < a1; a++) {
                const int i = __ffsll((long long)a) - 1;
                const uint64_t side = ((x >> i) & 1) ? ~x : x;
                cut += s_deg[i] - 2 * __popcll(s_adj[i] & side);
                x ^= 1ull << i;
                add_bin(h, cut, n_bins, bad);
            }
            if (bad) atomicOr(err, DERR_BAD_DESC);
        } else {
            // x = the chosen set; inside = edges within x, dsum = degrees summed
            // over x (k-vertex cover: dsum - inside edges touch x).  Between
            // consecutive states only the bits Gosper's step moves change:
            // removing r lowers inside by |N(r) & x|, adding v raises it by
            // |N(v) & x| (x without v).
            // y = the enumerated set (x itself, or its complement when
            // k > n/2), |y| = kk.  In increasing integer order the sets
            // {v} u T with v < min(T) have consecutive ranks, so a thread fixes
            // T, sweeps v, then moves T to its successor (Gosper).  With
            // I = inside(y) = inside(T) + |N(v) & T| and D = degree sum of y:
            //   DkS  x = y: I        x = ~y: m - D + I
            //   kVC  x = y: D - I    x = ~y: m - I
            const int kk = P.comp ? P.n - P.k : P.k;
            bool bad = false;
            if (kk == 0) {  // the single state: x = {} or x = all vertices
                const int c = P.comp ? P.m : 0;  // no edge inside / touching {}, all m for all vertices
                add_bin(h, c, n_bins, bad);
            } else {
                Set2 T = unrank_colex128(a0, P.n, kk, binom);
                int v = T.lo ? __ffsll((long long)T.lo) - 1 : 64 + __ffsll((long long)T.hi) - 1;
                if (v < 64) T.lo ^= 1ull << v;
                else T.hi ^= 1ull << (v - 64);
                const bool by_inside = (P.kind == 1) != (P.comp != 0);  // cost = I or m - I
                const bool packed = by_inside && kk <= 16;
                uint64_t rem = a1 - a0;
                for (;;) {
                    const int lim = T.lo ? __ffsll((long long)T.lo) - 1
                                         : (T.hi ? 64 + __ffsll((long long)T.hi) - 1 : P.n);
                    int tin = 0, tds = 0;
                    for (uint64_t z = T.lo; z; z &= z - 1) {
                        const int u = __ffsll((long long)z) - 1;
                        tin += __popcll(s_up_lo[u] & T.lo) + __popcll(s_up_hi[u] & T.hi);
                        tds += s_deg2[u];
                    }
                    for (uint64_t z = T.hi; z; z &= z - 1) {
                        const int u = 64 + __ffsll((long long)z) - 1;
                        tin += __popcll(s_up_lo[u] & T.lo) + __popcll(s_up_hi[u] & T.hi);
                        tds += s_deg2[u];
                    }
                    tin >>= 1;
                    const uint64_t span = lim > v ? (uint64_t)(lim - v) : 0ull;
                    const int cnt = (int)(span < rem ? span : rem);
                    if (packed) {
                        // |N(v) & T| < kk <= 16: counts in 8-bit fields (cnt < 128)
                        uint64_t f0 = 0, f1 = 0;
                        for (int i = 0; i < cnt; i++, v++) {
                            const int pv = __popcll(s_up_lo[v] & T.lo) + __popcll(s_up_hi[v] & T.hi);
                            if (pv < 8) f0 += 1ull << (8 * pv);
                            else f1 += 1ull << (8 * (pv - 8));
                        }
                        for (int f = 0; f < kk; f++) {
                            const uint32_t c = (uint32_t)(((f < 8 ? f0 : f1) >> (8 * (f & 7))) & 255u);
                            if (c) {
                                const int cost = P.comp ? P.m - (tin + f) : tin + f;
                                if ((unsigned)cost < (unsigned)n_bins) atomicAdd(&h[cost], c);
                                else bad = true;
                            }
                        }
                    } else {
                        for (int i = 0; i < cnt; i++, v++) {
                            const int I = tin + __popcll(s_up_lo[v] & T.lo) + __popcll(s_up_hi[v] & T.hi);
                            const int D = tds + s_deg2[v];
                            const int cost = P.kind == 1 ? (P.comp ? P.m - D + I : I) : (P.comp ? P.m - I : D - I);
                            add_bin(h, cost, n_bins, bad);
                        }
                    }
                    rem -= (uint64_t)cnt;
                    if (rem == 0 || kk == 1) break;
                    T = gosper_next(T);
                    v = 0;
                }
            }
            if (bad) atomicOr(err, DERR_BAD_DESC);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        unsigned long long s = 0;
        for (int c = 0; c < copies; c++) s += hist[(size_t)c * n_bins + b];
        if (s) atomicAdd(&counts[b], s);
    }
}

// ------------------------------------------------- bit-sliced weight-k count
// Weight-k problems whose cost is a function of I = |edges inside y| alone
// (densest k-subgraph with y = x, k-vertex cover with y = the complement),
// |y| = KK in 2..8.  The sets y = {v} u T with v < min(T) are counted per
// (KK-1)-set T at once: I = inside(T) + a(v) with a(v) = |N(v) & T|, and
// a(v) for all 128 vertices is the bitwise sum of the neighbour masks of T's
// members, held as three bit planes (a <= 7).  The histogram of a over
// v < min(T) is then a popcount per value of a.  T itself is T3 u {a, w}
// with w < a < min(T3): the planes of T3 are built once per T3 (a carry-save
// adder tree), those of T2 = T3 u {a} by one mask added per a, and those of T
// by one more per w.  A thread's change of T2 is then short, so the lanes of
// a warp, which change T2 at different times, stay together.  Threads take
// equal ranges of T's colex ranks, so every thread does the same work.
struct Planes {
    uint64_t b0l, b0h, b1l, b1h, b2l, b2h;
};

__device__ __forceinline__ void csa(uint64_t a, uint64_t b, uint64_t c, uint64_t &sum, uint64_t &carry) {
    sum = a ^ b ^ c;
    carry = (a & b) | (c & (a ^ b));
}

// a + m for one more mask m (no overflow: a <= 7 by construction)
__device__ __forceinline__ Planes planes_add(const Planes &P, uint64_t ml, uint64_t mh) {
    Planes Q;
    const uint64_t c0l = P.b0l & ml, c0h = P.b0h & mh;
    Q.b0l = P.b0l ^ ml;
    Q.b0h = P.b0h ^ mh;
    const uint64_t c1l = P.b1l & c0l, c1h = P.b1h & c0h;
    Q.b1l = P.b1l ^ c0l;
    Q.b1h = P.b1h ^ c0h;
    Q.b2l = P.b2l ^ c1l;
    Q.b2h = P.b2h ^ c1h;
    return Q;
}

__device__ __forceinline__ int lowest128(uint64_t lo, uint64_t hi, int none) {
    return lo ? __ffsll((long long)lo) - 1 : (hi ? 64 + __ffsll((long long)hi) - 1 : none);
}

// p[S] += the number of v whose plane bits include S (S = 1..7 as a set of
// planes); an S above KK - 1 has no v (every |N(v) & T| <= KK - 1).
template <int KK>
__device__ __forceinline__ void plane_popcounts(uint64_t x0, uint64_t x1, uint64_t x2, int (&p)[8]) {
#pragma unroll
    for (int S = 1; S < 8; S++) {
        if (S > KK - 1) continue;
        uint64_t m = ~0ull;
        if (S & 1) m &= x0;
        if (S & 2) m &= x1;
        if (S & 4) m &= x2;
        p[S] += __popcll(m);
    }
}

// The number of v with value exactly f, by inclusion-exclusion over the
// plane sets that contain f's bits.
template <int KK>
__device__ __forceinline__ int value_count(const int (&p)[8], int f) {
    int c = 0;
#pragma unroll
    for (int S = 1; S < 8; S++)
        if (S <= KK - 1 && (S & f) == f) c += (__popc((unsigned)(S ^ f)) & 1) ? -p[S] : p[S];
    return c;
}

template <int KK>
__global__ void __launch_bounds__(kDegThreads)
degeneracy_sliced_kernel(const DegParams P, const uint64_t *__restrict__ binom, uint64_t t_start, uint64_t t_count,
                         int n_bins, unsigned long long *__restrict__ counts, int *err) {
    constexpr int kNb = KK * (KK - 1) / 2 + 1;  // I = 0 .. C(KK, 2)
    extern __shared__ uint32_t hpriv[];          // [kNb][kDegThreads]: one column per thread
    __shared__ ulonglong2 s_up[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 128; i += blockDim.x) s_up[i] = make_ulonglong2(P.up_lo[i], P.up_hi[i]);
    for (int i = tid; i < kNb * kDegThreads; i += blockDim.x) hpriv[i] = 0u;
    __syncthreads();
    uint32_t *h = hpriv + tid;
    const int n = P.n;

    const uint64_t nthr = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + tid;
    const uint64_t per = (t_count + nthr - 1) / nthr;
    const uint64_t r0 = t_start + g * per;
    const uint64_t r1 = min(t_start + t_count, r0 + per);
    if (r0 < r1) {
        // T of rank r0 = T3 u {a, w}, w < a < min(T3); with KK = 2, T = {w}
        Set2 T3 = unrank_colex128(r0, n, KK - 1, binom);
        int w = lowest128(T3.lo, T3.hi, n);
        if (w < 64) T3.lo ^= 1ull << w;
        else T3.hi ^= 1ull << (w - 64);
        int a = n;
        if (KK >= 3) {
            a = lowest128(T3.lo, T3.hi, n);
            if (a < 64) T3.lo ^= 1ull << a;
            else T3.hi ^= 1ull << (a - 64);
        }
        Planes B3, B2;
        int tin3 = 0, lim3 = n, tin2 = 0;
        auto build_t3 = [&]() {
            // planes of |N(v) & T3| by a carry-save tree over T3's KK-3 members
            uint64_t ml[6], mh[6];
            uint64_t zl = T3.lo, zh = T3.hi;
#pragma unroll
            for (int j = 0; j < 6; j++) {
                ml[j] = mh[j] = 0ull;
                if (j < KK - 3) {
                    const int u = lowest128(zl, zh, 0);
                    if (u < 64) zl &= zl - 1;
                    else zh &= zh - 1;
                    const ulonglong2 m = s_up[u];
                    ml[j] = m.x;
                    mh[j] = m.y;
                }
            }
            uint64_t s1l, c1l, s2l, c2l, s1h, c1h, s2h, c2h;
            csa(ml[0], ml[1], ml[2], s1l, c1l);
            csa(ml[3], ml[4], ml[5], s2l, c2l);
            csa(mh[0], mh[1], mh[2], s1h, c1h);
            csa(mh[3], mh[4], mh[5], s2h, c2h);
            B3.b0l = s1l ^ s2l;
            B3.b0h = s1h ^ s2h;
            csa(c1l, c2l, s1l & s2l, B3.b1l, B3.b2l);
            csa(c1h, c2h, s1h & s2h, B3.b1h, B3.b2h);
            // inside(T3) = (sum over members u of |N(u) & T3|) / 2
            tin3 = (__popcll(B3.b0l & T3.lo) + __popcll(B3.b0h & T3.hi) +
                    2 * (__popcll(B3.b1l & T3.lo) + __popcll(B3.b1h & T3.hi)) +
                    4 * (__popcll(B3.b2l & T3.lo) + __popcll(B3.b2h & T3.hi))) >> 1;
            lim3 = KK >= 4 ? lowest128(T3.lo, T3.hi, n) : n;
        };
        // T2 = T3 u {a}: one more mask, inside(T2) = inside(T3) + |N(a) & T3|
        auto set_t2 = [&]() {
            if (KK >= 3) {
                const ulonglong2 m = s_up[a];
                B2 = planes_add(B3, m.x, m.y);
                tin2 = tin3 + __popcll(m.x & T3.lo) + __popcll(m.y & T3.hi);
            } else {
                B2 = B3;
                tin2 = 0;
            }
        };
        build_t3();
        set_t2();
        for (uint64_t r = r0; r < r1; r++) {
            // T = T2 u {w}: its planes, inside(T) = inside(T2) + a_T2(w), and
            // the planes' popcounts over v < w
            int p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            int aw;
            if (w < 64) {  // every v < w in the low word (nearly every T)
                const uint64_t ml = s_up[w].x, R = (1ull << w) - 1ull;
                const uint64_t c0 = B2.b0l & ml, c1 = B2.b1l & c0;
                plane_popcounts<KK>((B2.b0l ^ ml) & R, (B2.b1l ^ c0) & R, (B2.b2l ^ c1) & R, p);
                aw = (int)((B2.b0l >> w) & 1ull) + 2 * (int)((B2.b1l >> w) & 1ull) + 4 * (int)((B2.b2l >> w) & 1ull);
            } else {
                const ulonglong2 m = s_up[w];
                const Planes B = planes_add(B2, m.x, m.y);
                const uint64_t Rh = (1ull << (w - 64)) - 1ull;
                plane_popcounts<KK>(B.b0l, B.b1l, B.b2l, p);
                plane_popcounts<KK>(B.b0h & Rh, B.b1h & Rh, B.b2h & Rh, p);
                const int sh = w - 64;
                aw = (int)((B2.b0h >> sh) & 1ull) + 2 * (int)((B2.b1h >> sh) & 1ull) + 4 * (int)((B2.b2h >> sh) & 1ull);
            }
            const int tin = tin2 + aw;
            int rest = w;
#pragma unroll
            for (int f = 1; f < KK; f++) {
                const int c = value_count<KK>(p, f);
                rest -= c;
                h[(tin + f) * kDegThreads] += (uint32_t)c;
            }
            h[tin * kDegThreads] += (uint32_t)rest;
            // next T: w + 1 below a, else a + 1 below min(T3), else the next
            // T3 with at least two vertices below it (a >= 1 and w < a)
            if (++w >= a && KK >= 3 && r + 1 < r1) {
                w = 0;
                if (++a >= lim3) {
                    if (KK >= 4) {
                        do {
                            T3 = gosper_next(T3);
                            build_t3();
                        } while (lim3 < 2);
                    }
                    a = 1;
                }
                set_t2();
            }
        }
    }
    __syncthreads();
    // bins: one warp per value of I, fixed order
    for (int I = warp; I < kNb; I += kDegWarps) {
        unsigned long long sacc = 0;
        for (int t = lane; t < kDegThreads; t += 32) sacc += hpriv[I * kDegThreads + t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
        if (lane == 0 && sacc) {
            const int cost = P.kind == 1 ? I : P.m - I;
            if ((unsigned)cost < (unsigned)n_bins) atomicAdd(&counts[cost], sacc);
            else atomicOr(err, DERR_BAD_DESC);
        }
    }
}

// ------------------------------------------------------- reduced simulation
// One CTA per angle set, as many threads as values (a warp at least, 512 at
// most).  Float64 runs at a small fraction of the float32 rate here, so the
// per-value constants sqrt(d_j / N) and the mixer's cos / sin are computed
// once per set, not in every loop.
constexpr int kGrMaxThreads = 512;
constexpr int kGrMaxWarps = kGrMaxThreads / 32;

// Deterministic block sum of a complex float64 (fixed reduction order);
// every thread gets the total.
__device__ double2 block_sum2(double2 v, double2 *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int nw = blockDim.x >> 5;
    if (nw == 1) return v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < nw; w++) {
        t.x += red[w].x;
        t.y += red[w].y;
    }
    return t;
}

__device__ __forceinline__ double2 cmuld(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(kGrMaxThreads)
grover_eval_kernel(const int64_t *__restrict__ counts, int nb, int p, const double *__restrict__ angles,
                   double *__restrict__ E, double *__restrict__ grad) {
    extern __shared__ double2 gsm[];
    double2 *psi = gsm, *lam = gsm + nb, *red = gsm + 2 * nb, *trig = red + kGrMaxWarps;
    double *u = reinterpret_cast<double *>(trig + p);
    const int set = blockIdx.x;
    const double *a = angles + (size_t)set * 2 * p;
    // N = sum of the degeneracies (exact in float64 below 2^53)
    double2 nn = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) nn.x += (double)counts[j];
    const double N = block_sum2(nn, red).x;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        u[j] = sqrt((double)counts[j] / N);
        psi[j] = make_double2(u[j], 0.0);
    }
    for (int k = threadIdx.x; k < p; k += blockDim.x) {
        double sb, cb;
        sincos(a[k], &sb, &cb);
        trig[k] = make_double2(cb, sb);
    }
    __syncthreads();
    for (int k = 0; k < p; k++) {
        const double g = a[p + k];
        double2 s = make_double2(0.0, 0.0);
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            double sn, cs;
            sincos(g * (double)j, &sn, &cs);
            psi[j] = cmuld(psi[j], make_double2(cs, -sn));
            s.x += u[j] * psi[j].x;
            s.y += u[j] * psi[j].y;
        }
        s = block_sum2(s, red);
        const double2 d = cmuld(make_double2(trig[k].x - 1.0, -trig[k].y), s);  // (e^{-i b} - 1) <u|psi>
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            psi[j].x += d.x * u[j];
            psi[j].y += d.y * u[j];
        }
    }
    double2 e = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) e.x += (double)j * (psi[j].x * psi[j].x + psi[j].y * psi[j].y);
    e = block_sum2(e, red);
    if (threadIdx.x == 0) E[set] = e.x;
    if (!grad) return;
    double *g_out = grad + (size_t)set * 2 * p;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) lam[j] = make_double2((double)j * psi[j].x, (double)j * psi[j].y);
    for (int k = p - 1; k >= 0; k--) {
        const double g = a[p + k];
        double2 sl = make_double2(0.0, 0.0), sp = make_double2(0.0, 0.0);
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            sl.x += u[j] * lam[j].x;
            sl.y += u[j] * lam[j].y;
            sp.x += u[j] * psi[j].x;
            sp.y += u[j] * psi[j].y;
        }
        sl = block_sum2(sl, red);
        sp = block_sum2(sp, red);
        // dE/dbeta_k = 2 Im( conj(<u|lam>) <u|psi> )
        if (threadIdx.x == 0) g_out[k] = 2.0 * (sl.x * sp.y - sl.y * sp.x);
        const double2 f = make_double2(trig[k].x - 1.0, trig[k].y);  // e^{+i b} - 1
        const double2 dl = cmuld(f, sl), dp = cmuld(f, sp);
        double2 gg = make_double2(0.0, 0.0);
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            lam[j].x += dl.x * u[j];
            lam[j].y += dl.y * u[j];
            psi[j].x += dp.x * u[j];
            psi[j].y += dp.y * u[j];
            // Im( conj(lam_j) c_j psi_j )
            gg.x += (double)j * (lam[j].x * psi[j].y - lam[j].y * psi[j].x);
            double sn, cs;
            sincos(g * (double)j, &sn, &cs);
            const double2 ph = make_double2(cs, sn);
            lam[j] = cmuld(lam[j], ph);
            psi[j] = cmuld(psi[j], ph);
        }
        gg = block_sum2(gg, red);
        if (threadIdx.x == 0) g_out[p + k] = 2.0 * gg.x;
    }
}

}  // namespace

int grover_max_bins() { return 4096; }

static DegParams deg_params(const DegLaunch &L) {
    DegParams P;
    memset(&P, 0, sizeof(P));
    for (int i = 0; i < 128; i++) {
        P.up_lo[i] = L.up_lo[i];
        P.up_hi[i] = L.up_hi[i];
    }
    for (int i = 0; i < 64; i++) {
        P.adj[i] = L.adj[i];
        P.deg[i] = L.deg[i];
    }
    P.n = L.n;
    P.k = L.k;
    P.m = L.m;
    P.kind = L.kind;
    P.comp = L.comp;
    return P;
}

int degeneracy_sliced_kk(const DegLaunch &L) {
    if (L.kind == 0) return 0;
    const int kk = L.comp ? L.n - L.k : L.k;
    const bool by_inside = (L.kind == 1) != (L.comp != 0);  // cost = I (DkS) or m - I (cover, complement)
    return by_inside && kk >= 2 && kk <= 8 ? kk : 0;
}

template <int KK>
static cudaError_t go_sliced(const DegParams &P, const uint64_t *d_binom, uint64_t t_start, uint64_t t_count,
                             int n_bins, unsigned long long *d_counts, int *d_err, cudaStream_t s) {
    constexpr int nb = KK * (KK - 1) / 2 + 1;
    const size_t smem = (size_t)nb * kDegThreads * 4;
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, degeneracy_sliced_kernel<KK>, kDegThreads,
                                                                  smem);
    if (e != cudaSuccess) return e;
    const uint64_t want = (t_count + (uint64_t)kDegThreads * 8 - 1) / ((uint64_t)kDegThreads * 8);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)nsm * std::max(1, occ)));
    degeneracy_sliced_kernel<KK><<<grid, kDegThreads, smem, s>>>(P, d_binom, t_start, t_count, n_bins, d_counts,
                                                                 d_err);
    return cudaGetLastError();
}

cudaError_t launch_degeneracy_sliced(const DegLaunch &L, const uint64_t *d_binom, uint64_t t_start,
                                     uint64_t t_count, unsigned long long *d_counts, int *d_err, cudaStream_t s) {
    const DegParams P = deg_params(L);
    switch (degeneracy_sliced_kk(L)) {
    case 2: return go_sliced<2>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 3: return go_sliced<3>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 4: return go_sliced<4>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 5: return go_sliced<5>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 6: return go_sliced<6>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 7: return go_sliced<7>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    case 8: return go_sliced<8>(P, d_binom, t_start, t_count, L.n_bins, d_counts, d_err, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_degeneracy(const DegLaunch &L, const uint64_t *d_binom, uint64_t start, uint64_t count,
                              unsigned long long *d_counts, int *d_err, cudaStream_t s) {
    DegParams P = deg_params(L);
    int copies = (96 * 1024) / (4 * L.n_bins);
    copies = std::max(1, std::min(kDegWarps, copies));
    const size_t smem = (size_t)copies * L.n_bins * 4;
    static int attr_done[kMaxDevices];
    {
        cudaError_t e = smem_attr_once(degeneracy_kernel, 96 * 1024 + 4 * 4096, attr_done);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (count + (uint64_t)kDegThreads * 64 - 1) / ((uint64_t)kDegThreads * 64);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)nsm * 8));
    degeneracy_kernel<<<grid, kDegThreads, smem, s>>>(P, d_binom, start, count, L.n_bins, copies, d_counts, d_err);
    return cudaGetLastError();
}

cudaError_t launch_grover_eval(const int64_t *d_counts, int nb, int p, int n_sets, const double *d_angles,
                               double *d_E, double *d_grad, cudaStream_t s) {
    const size_t smem = (size_t)(2 * nb + kGrMaxWarps + p) * sizeof(double2) + (size_t)nb * sizeof(double);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    static int attr_done[kMaxDevices];
    {
        cudaError_t e = smem_attr_once(grover_eval_kernel, 200 * 1024, attr_done);
        if (e != cudaSuccess) return e;
    }
    const int threads = std::min(kGrMaxThreads, std::max(32, (nb + 31) / 32 * 32));
    grover_eval_kernel<<<n_sets, threads, smem, s>>>(d_counts, nb, p, d_angles, d_E, d_grad);
    return cudaGetLastError();
}

}  // namespace qg
