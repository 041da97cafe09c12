/*
 * CPU oracle for direct statevector QAOA simulation (arXiv 2312.06451,
 * "JuliQAOA: Fast, Flexible QAOA Simulation").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or constant with the CUDA library, and it includes
 * nothing from it.
 *
 * Everything runs in complex128 / float64, one amplitude at a time, in the
 * order the paper states the method:
 *
 *   state   |beta,gamma> = e^{-i b_p H_M} e^{-i g_p H_C} ... e^{-i b_1 H_M}
 *                          e^{-i g_1 H_C} |psi_0>                  (Eq. 1)
 *   target  <C> = <beta,gamma| C |beta,gamma>                      (Sec. 1)
 *   H_C|x>  = C(x)|x>, C stored over the feasible set S            (Sec. 2.1)
 *   X mixer H_M = sum_i X_i, applied as one 2x2 rotation per qubit
 *           (a sequence of single-qubit operations, Sec. 2.2; Eq. 2 is the
 *           equivalent Hadamard-diagonal form, checked separately in tests)
 *   ring mixer H_M = sum_i (X_i X_{i+1} + Y_i Y_{i+1}) restricted to the
 *           Hamming-weight-k subspace (Sec. 2.1), exponentiated directly by
 *           its power series (no eigendecomposition, so it is independent of
 *           the V D V^-1 route the GPU path takes)
 *   angles  [beta_1..beta_p, gamma_1..gamma_p]                     (Listing 1)
 *   default psi_0 = uniform superposition over S                   (Sec. 3)
 *   gradient: exact reverse mode (the adjoint recurrences; Sec. 2.3 and
 *           Sec. 4 describe gradients by reverse-mode automatic
 *           differentiation) in complex128, undoing each unitary exactly.
 *
 * Readings of points the paper leaves open (bit order, ring wrap-around,
 * SK spin convention, Dicke ordering) are stated at each function.
 *
 * Parity pins: every function here is pinned by tests that do not reuse its
 * arithmetic (dense matrix exponentials, the p=1 MaxCut closed form, sum
 * rules, symmetries, free-fermion ring spectrum, finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { ORACLE_MIXER_X = 0, ORACLE_MIXER_RING = 1, ORACLE_MIXER_CLIQUE = 2, ORACLE_MIXER_GROVER = 3 };

/* ------------------------------------------------------------------ threads */

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* --------------------------------------------------------- feasible states */

/* Hamming-weight-k basis states of n qubits, in increasing integer order
 * (Sec. 2.1 feasible subspace of size binom(n,k); Sec. 2.4 enumerates them in
 * increasing order with Gosper's hack).  Plain scan over all 2^n integers.
 * Bit i of a state is qubit i.  Returns the count; writes it to out if
 * out != NULL. */
int64_t oracle_dicke_states(int n, int k, uint64_t *out) {
    int64_t cnt = 0;
    for (uint64_t x = 0; x < ((uint64_t)1 << n); x++) {
        if (__builtin_popcountll(x) == k) {
            if (out) out[cnt] = x;
            cnt++;
        }
    }
    return cnt;
}

static inline uint64_t state_at(const uint64_t *states, int64_t a) {
    return states ? states[a] : (uint64_t)a;
}

static inline int bit(uint64_t x, int i) { return (int)((x >> i) & 1u); }

/* ------------------------------------------------------------ cost vectors */

/* MaxCut (Sec. 3, Listing 1): C(x) = sum over edges (u,v) of w_uv [x_u != x_v],
 * w = 1 when weights == NULL.  Evaluated on states[0..dim) (all 2^n integers
 * when states == NULL). */
void oracle_cost_maxcut(int n, int m, const int32_t *edges, const double *weights,
                        int64_t dim, const uint64_t *states, double *out) {
    (void)n;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < dim; a++) {
        uint64_t x = state_at(states, a);
        double c = 0.0;
        for (int e = 0; e < m; e++) {
            int u = edges[2 * e], v = edges[2 * e + 1];
            if (bit(x, u) != bit(x, v)) c += weights ? weights[e] : 1.0;
        }
        out[a] = c;
    }
}

/* Sherrington-Kirkpatrick cost, an arbitrary user cost (Sec. 3: any function
 * of the basis state is accepted): C(x) = sum_{i<j} J_ij z_i z_j with the
 * spin z_i = 1 - 2 x_i.  J is a row-major n x n matrix; only i < j is read. */
void oracle_cost_sk(int n, const double *J, int64_t dim, const uint64_t *states,
                    double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < dim; a++) {
        uint64_t x = state_at(states, a);
        double c = 0.0;
        for (int i = 0; i < n; i++) {
            double zi = 1.0 - 2.0 * bit(x, i);
            for (int j = i + 1; j < n; j++) {
                double zj = 1.0 - 2.0 * bit(x, j);
                c += J[i * n + j] * zi * zj;
            }
        }
        out[a] = c;
    }
}

/* Densest k-subgraph (Sec. 2.1, Listing 2): number of edges with both
 * endpoints selected, C(x) = sum over edges [x_u = 1 and x_v = 1]. */
void oracle_cost_dks(int n, int m, const int32_t *edges, int64_t dim,
                     const uint64_t *states, double *out) {
    (void)n;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < dim; a++) {
        uint64_t x = state_at(states, a);
        double c = 0.0;
        for (int e = 0; e < m; e++)
            if (bit(x, edges[2 * e]) && bit(x, edges[2 * e + 1])) c += 1.0;
        out[a] = c;
    }
}

/* Max k-vertex cover (Sec. 2.1, a Hamming-weight-k problem): number of edges
 * with at least one endpoint selected. */
void oracle_cost_kvc(int n, int m, const int32_t *edges, int64_t dim,
                     const uint64_t *states, double *out) {
    (void)n;
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < dim; a++) {
        uint64_t x = state_at(states, a);
        double c = 0.0;
        for (int e = 0; e < m; e++)
            if (bit(x, edges[2 * e]) || bit(x, edges[2 * e + 1])) c += 1.0;
        out[a] = c;
    }
}

/* ---------------------------------------------------------------- mixers */

typedef struct {
    int kind;               /* ORACLE_MIXER_X, _RING, _CLIQUE or _GROVER */
    int n;
    int64_t dim;
    const uint64_t *states; /* ring, clique: the sorted Hamming-weight-k states */
} mixer_t;

/* Position of state s in the sorted feasible list (binary search). */
static int64_t find_state(const mixer_t *mx, uint64_t s) {
    int64_t lo = 0, hi = mx->dim - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        uint64_t v = mx->states[mid];
        if (v == s) return mid;
        if (v < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* out = H_M v.
 * X mixer: (sum_i X_i v)_x = sum_i v_{x xor 2^i}.
 * Ring mixer (Sec. 2.1): sum over ring edges (i, i+1 mod n) of
 * X_i X_j + Y_i Y_j.  On two qubits this operator maps |01> <-> |10> with
 * matrix element 2 and annihilates |00>, |11>; so on a basis state it swaps
 * bits i and j with weight 2 when they differ.  The ring is read as periodic
 * (edge n-1 -- 0 included), coefficient 1 per edge.
 * Clique mixer (Sec. 2.1): the same two-qubit term on every pair i < j.
 * Grover mixer (Sec. 2.4): H_G = |u><u| with u the uniform superposition over
 * the feasible set, so (H_G v)_a = (sum_b v_b) / dim. */
static void hm_apply(const mixer_t *mx, const cplx *v, cplx *out) {
    const int n = mx->n;
    if (mx->kind == ORACLE_MIXER_GROVER) {
        cplx s = 0.0;
        for (int64_t a = 0; a < mx->dim; a++) s += v[a];
        for (int64_t a = 0; a < mx->dim; a++) out[a] = s / (double)mx->dim;
        return;
    }
    if (mx->kind == ORACLE_MIXER_X) {
#pragma omp parallel for schedule(static)
        for (int64_t x = 0; x < mx->dim; x++) {
            cplx s = 0.0;
            for (int i = 0; i < n; i++) s += v[x ^ ((int64_t)1 << i)];
            out[x] = s;
        }
    } else if (mx->kind == ORACLE_MIXER_CLIQUE) {
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < mx->dim; a++) {
            uint64_t x = mx->states[a];
            cplx s = 0.0;
            for (int i = 0; i < n; i++)
                for (int j = i + 1; j < n; j++)
                    if (bit(x, i) != bit(x, j)) {
                        uint64_t y = x ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                        s += 2.0 * v[find_state(mx, y)];
                    }
            out[a] = s;
        }
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < mx->dim; a++) {
            uint64_t x = mx->states[a];
            cplx s = 0.0;
            for (int i = 0; i < n; i++) {
                int j = (i + 1) % n;
                if (bit(x, i) != bit(x, j)) {
                    uint64_t y = x ^ ((uint64_t)1 << i) ^ ((uint64_t)1 << j);
                    s += 2.0 * v[find_state(mx, y)];
                }
            }
            out[a] = s;
        }
    }
}

/* v <- e^{-i beta H_M} v.
 * X mixer: the X_i commute, so e^{-i beta sum X_i} = prod_i e^{-i beta X_i};
 * e^{-i beta X} = cos(beta) I - i sin(beta) X acts on each amplitude pair
 * (x, x xor 2^i) (Sec. 2.2: a sequence of single-qubit operations).
 * Ring and clique mixers: the exponential series sum_j (-i tau H)^j / j!
 * applied to v, with beta split into s equal steps tau so that
 * |tau| * ||H|| <= 1/2; the series is summed until its terms fall below 1e-18
 * of the running sum.  ||H|| <= max row sum: 2n for the ring, 2 k (n - k)
 * for the clique (a weight-k state has k (n - k) pairs of differing bits). */
static void mixer_apply(const mixer_t *mx, double beta, cplx *v, cplx *tmp1, cplx *tmp2) {
    const int64_t dim = mx->dim;
    if (mx->kind == ORACLE_MIXER_GROVER) {
        /* H_G is a projector: e^{-i beta H_G} = I + (e^{-i beta} - 1) |u><u| */
        cplx s = 0.0;
        for (int64_t a = 0; a < dim; a++) s += v[a];
        const cplx d = (cexp(-I * beta) - 1.0) * s / (double)dim;
        for (int64_t a = 0; a < dim; a++) v[a] += d;
        return;
    }
    if (mx->kind == ORACLE_MIXER_X) {
        const double c = cos(beta), s = sin(beta);
        for (int i = 0; i < mx->n; i++) {
            const int64_t st = (int64_t)1 << i;
#pragma omp parallel for schedule(static)
            for (int64_t j = 0; j < dim / 2; j++) {
                int64_t lo = j & (st - 1);
                int64_t x0 = ((j - lo) << 1) | lo; /* bit i of x0 is 0 */
                int64_t x1 = x0 | st;
                cplx a = v[x0], b = v[x1];
                v[x0] = c * a - I * s * b;
                v[x1] = -I * s * a + c * b;
            }
        }
        return;
    }
    double hnorm = 2.0 * mx->n;
    if (mx->kind == ORACLE_MIXER_CLIQUE) {
        const int k = __builtin_popcountll(mx->states[0]);
        hnorm = 2.0 * k * (mx->n - k);
        if (hnorm < 1.0) hnorm = 1.0;
    }
    int steps = (int)ceil(fabs(beta) * hnorm / 0.5);
    if (steps < 1) steps = 1;
    const double tau = beta / steps;
    cplx *term = tmp1, *hterm = tmp2;
    for (int st = 0; st < steps; st++) {
        memcpy(term, v, sizeof(cplx) * dim);
        for (int j = 1; j < 80; j++) {
            hm_apply(mx, term, hterm);
            double tmax = 0.0, vmax = 0.0;
            for (int64_t a = 0; a < dim; a++) {
                term[a] = (-I * tau / j) * hterm[a];
                v[a] += term[a];
                if (cabs(term[a]) > tmax) tmax = cabs(term[a]);
                if (cabs(v[a]) > vmax) vmax = cabs(v[a]);
            }
            if (tmax <= 1e-18 * vmax) break;
        }
    }
}

/* v <- e^{-i gamma H_C} v, i.e. v_x <- e^{-i gamma C(x)} v_x (Eq. 1). */
static void phase_apply(int64_t dim, const double *cost, double gamma, cplx *v) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < dim; a++) v[a] *= cexp(-I * gamma * cost[a]);
}

static void init_state(int64_t dim, const double *psi0, cplx *v) {
    if (psi0) {
        for (int64_t a = 0; a < dim; a++) v[a] = psi0[2 * a] + I * psi0[2 * a + 1];
    } else {
        const double amp = 1.0 / sqrt((double)dim);
        for (int64_t a = 0; a < dim; a++) v[a] = amp;
    }
}

static int make_mixer(mixer_t *mx, int kind, int n, int64_t dim, const uint64_t *states) {
    mx->kind = kind; mx->n = n; mx->dim = dim; mx->states = states;
    if (kind == ORACLE_MIXER_X) return dim == ((int64_t)1 << n) ? 0 : -1;
    if (kind == ORACLE_MIXER_RING) return (states && n >= 3) ? 0 : -1;
    if (kind == ORACLE_MIXER_CLIQUE) return (states && n >= 2 && dim >= 1) ? 0 : -1;
    if (kind == ORACLE_MIXER_GROVER) return dim >= 1 ? 0 : -1;
    return -1;
}

/* ------------------------------------------------------------ simulation */

/* Final state of Eq. 1: for k = 1..p apply the phase separator with gamma_k,
 * then the mixer with beta_k.  psi0 (interleaved re,im) may be NULL for the
 * uniform superposition over the feasible set.  psi_out is interleaved. */
int oracle_qaoa_state(int kind, int n, int64_t dim, const uint64_t *states,
                      const double *cost, int p, const double *angles,
                      const double *psi0, double *psi_out) {
    mixer_t mx;
    if (make_mixer(&mx, kind, n, dim, states) || p < 0) return -1;
    cplx *v = (cplx *)psi_out;
    cplx *t1 = NULL, *t2 = NULL;
    if (kind != ORACLE_MIXER_X) {
        t1 = malloc(sizeof(cplx) * dim); t2 = malloc(sizeof(cplx) * dim);
        if (!t1 || !t2) { free(t1); free(t2); return -2; }
    }
    init_state(dim, psi0, v);
    for (int k = 0; k < p; k++) {
        phase_apply(dim, cost, angles[p + k], v);
        mixer_apply(&mx, angles[k], v, t1, t2);
    }
    free(t1); free(t2);
    return 0;
}

static double expect(int64_t dim, const double *cost, const cplx *v) {
    double e = 0.0;
#pragma omp parallel for reduction(+ : e) schedule(static)
    for (int64_t a = 0; a < dim; a++) {
        double pr = creal(v[a]) * creal(v[a]) + cimag(v[a]) * cimag(v[a]);
        e += pr * cost[a];
    }
    return e;
}

/* <C> = sum_x |psi_x|^2 C(x) on the final state of Eq. 1.  Returns NAN on a
 * bad argument or an allocation failure. */
double oracle_qaoa_expectation(int kind, int n, int64_t dim, const uint64_t *states,
                               const double *cost, int p, const double *angles,
                               const double *psi0) {
    double *buf = malloc(sizeof(double) * 2 * dim);
    if (!buf) return NAN;
    if (oracle_qaoa_state(kind, n, dim, states, cost, p, angles, psi0, buf)) {
        free(buf);
        return NAN;
    }
    double e = expect(dim, cost, (const cplx *)buf);
    free(buf);
    return e;
}

/* <C> and all 2p partial derivatives, by exact reverse mode.
 *
 * Forward: psi_p from Eq. 1.  Backward, with lam = C psi_p and psi = psi_p:
 *   for k = p..1:
 *     dE/dbeta_k  = 2 Im <lam| H_M |psi>
 *     lam <- e^{+i beta_k H_M} lam,  psi <- e^{+i beta_k H_M} psi
 *     dE/dgamma_k = 2 Im <lam| C |psi>
 *     lam <- e^{+i gamma_k C} lam,   psi <- e^{+i gamma_k C} psi
 * (E = <psi_p|C|psi_p>; differentiating the unitary e^{-i t A} gives -iA, and
 * 2 Re <lam| -i A psi> = 2 Im <lam|A|psi>.)  Undoing a unitary is applying it
 * with the negated angle.  grad has the angle layout of Listing 1. */
int oracle_qaoa_gradient(int kind, int n, int64_t dim, const uint64_t *states,
                         const double *cost, int p, const double *angles,
                         const double *psi0, double *E, double *grad) {
    mixer_t mx;
    if (make_mixer(&mx, kind, n, dim, states) || p < 1) return -1;
    cplx *psi = malloc(sizeof(cplx) * dim);
    cplx *lam = malloc(sizeof(cplx) * dim);
    cplx *hv = malloc(sizeof(cplx) * dim);
    cplx *t2 = kind != ORACLE_MIXER_X ? malloc(sizeof(cplx) * dim) : NULL;
    if (!psi || !lam || !hv || (kind != ORACLE_MIXER_X && !t2)) {
        free(psi); free(lam); free(hv); free(t2);
        return -2;
    }
    cplx *t1 = lam; /* scratch for the ring series during the forward sweep */
    init_state(dim, psi0, psi);
    for (int k = 0; k < p; k++) {
        phase_apply(dim, cost, angles[p + k], psi);
        mixer_apply(&mx, angles[k], psi, t1, t2);
    }
    *E = expect(dim, cost, psi);
    for (int64_t a = 0; a < dim; a++) lam[a] = cost[a] * psi[a];

    for (int k = p - 1; k >= 0; k--) {
        hm_apply(&mx, psi, hv);
        double gb = 0.0;
#pragma omp parallel for reduction(+ : gb) schedule(static)
        for (int64_t a = 0; a < dim; a++) gb += cimag(conj(lam[a]) * hv[a]);
        grad[k] = 2.0 * gb;
        /* scratch for the ring series: hv is free again */
        mixer_apply(&mx, -angles[k], lam, hv, t2);
        mixer_apply(&mx, -angles[k], psi, hv, t2);
        double gg = 0.0;
#pragma omp parallel for reduction(+ : gg) schedule(static)
        for (int64_t a = 0; a < dim; a++) gg += cimag(conj(lam[a]) * cost[a] * psi[a]);
        grad[p + k] = 2.0 * gg;
        phase_apply(dim, cost, -angles[p + k], lam);
        phase_apply(dim, cost, -angles[p + k], psi);
    }
    free(psi); free(lam); free(hv); free(t2);
    return 0;
}

/* ------------------------------------------------------ multi-angle QAOA */

/* Multi-angle QAOA (Sec. 3: several mixers per layer, each with its own
 * angle): round k applies e^{-i gamma_k C}, then e^{-i beta_{k,q} X_q} for every
 * qubit q (the X_q commute, so their order does not matter).  Angles:
 * beta_{k,q} = angles[k n + q] (k < p, q < n), gamma_k = angles[p n + k];
 * grad has the same layout.  X mixer on all 2^n states only.  Reverse mode
 * as in oracle_qaoa_gradient, with one partial per (round, qubit):
 *   dE/dbeta_{k,q} = 2 Im <lam| X_q |psi>. */
static void rot_qubit(int64_t dim, int q, double beta, cplx *v) {
    const double c = cos(beta), s = sin(beta);
    const int64_t st = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < dim / 2; j++) {
        int64_t lo = j & (st - 1);
        int64_t x0 = ((j - lo) << 1) | lo, x1 = x0 | st;
        cplx a = v[x0], b = v[x1];
        v[x0] = c * a - I * s * b;
        v[x1] = -I * s * a + c * b;
    }
}

int oracle_qaoa_gradient_ma(int n, const double *cost, int p, const double *angles,
                            const double *psi0, double *E, double *grad) {
    const int64_t dim = (int64_t)1 << n;
    if (p < 1 || n < 1 || n > 30) return -1;
    cplx *psi = malloc(sizeof(cplx) * dim);
    cplx *lam = malloc(sizeof(cplx) * dim);
    if (!psi || !lam) { free(psi); free(lam); return -2; }
    init_state(dim, psi0, psi);
    for (int k = 0; k < p; k++) {
        phase_apply(dim, cost, angles[p * n + k], psi);
        for (int q = 0; q < n; q++) rot_qubit(dim, q, angles[k * n + q], psi);
    }
    *E = expect(dim, cost, psi);
    for (int64_t a = 0; a < dim; a++) lam[a] = cost[a] * psi[a];
    for (int k = p - 1; k >= 0; k--) {
        for (int q = 0; q < n; q++) {
            const int64_t st = (int64_t)1 << q;
            double gb = 0.0;
#pragma omp parallel for reduction(+ : gb) schedule(static)
            for (int64_t a = 0; a < dim; a++) gb += cimag(conj(lam[a]) * psi[a ^ st]);
            grad[k * n + q] = 2.0 * gb;
        }
        for (int q = 0; q < n; q++) {
            rot_qubit(dim, q, -angles[k * n + q], lam);
            rot_qubit(dim, q, -angles[k * n + q], psi);
        }
        double gg = 0.0;
#pragma omp parallel for reduction(+ : gg) schedule(static)
        for (int64_t a = 0; a < dim; a++) gg += cimag(conj(lam[a]) * cost[a] * psi[a]);
        grad[p * n + k] = 2.0 * gg;
        phase_apply(dim, cost, -angles[p * n + k], lam);
        phase_apply(dim, cost, -angles[p * n + k], psi);
    }
    free(psi); free(lam);
    return 0;
}

/* ----------------------------------------- general X mixers (Sec. 2.1) */

/* Mixers written as sums of products of Pauli X: H_M = f(X) with
 * f(X) = sum_S c_{|S|} prod_{i in S} X_i (Sec. 2.1: e^{-i beta f(X_i)} =
 * H^n e^{-i beta f(Z_i)} H^n, with the diagonal form precomputed).  On the
 * Hadamard-basis state |z> of weight w, prod_{i in S} Z_i has eigenvalue
 * (-1)^{|S & z|}, so f(Z) = d_w with d_w = sum_k c_k K_k(w), K_k the
 * Krawtchouk polynomial sum_j (-1)^j C(w, j) C(n - w, k - j).  The oracle
 * takes d[0..n] and applies e^{-i beta H_M} literally: a Walsh-Hadamard
 * transform (n Hadamard butterflies), the weight phases, the transform again.
 * The Grover mixer |+><+| is c_k = 2^-n for all k, i.e. d_w = [w = 0]. */
static void hadamard_all(int n, cplx *v) {
    const int64_t dim = (int64_t)1 << n;
    const double r = 1.0 / sqrt(2.0);
    for (int q = 0; q < n; q++) {
        const int64_t st = (int64_t)1 << q;
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < dim / 2; j++) {
            int64_t lo = j & (st - 1);
            int64_t x0 = ((j - lo) << 1) | lo, x1 = x0 | st;
            cplx a = v[x0], b = v[x1];
            v[x0] = r * (a + b);
            v[x1] = r * (a - b);
        }
    }
}

static void general_mixer(int n, const double *d, double beta, cplx *v) {
    const int64_t dim = (int64_t)1 << n;
    hadamard_all(n, v);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < dim; x++) v[x] *= cexp(-I * beta * d[__builtin_popcountll((uint64_t)x)]);
    hadamard_all(n, v);
}

/* out = H_M v = H^n diag(d_w) H^n v. */
static void general_hm(int n, const double *d, const cplx *v, cplx *out) {
    const int64_t dim = (int64_t)1 << n;
    memcpy(out, v, sizeof(cplx) * dim);
    hadamard_all(n, out);
    for (int64_t x = 0; x < dim; x++) out[x] *= d[__builtin_popcountll((uint64_t)x)];
    hadamard_all(n, out);
}

/* <C> and its 2p derivatives (angle layout of Listing 1) for the general X
 * mixer with Hadamard-basis weights d[0..n]; reverse mode as in
 * oracle_qaoa_gradient. */
int oracle_qaoa_gradient_general(int n, const double *d, const double *cost, int p, const double *angles,
                                 const double *psi0, double *E, double *grad) {
    const int64_t dim = (int64_t)1 << n;
    if (p < 1 || n < 1 || n > 30) return -1;
    cplx *psi = malloc(sizeof(cplx) * dim), *lam = malloc(sizeof(cplx) * dim), *hv = malloc(sizeof(cplx) * dim);
    if (!psi || !lam || !hv) { free(psi); free(lam); free(hv); return -2; }
    init_state(dim, psi0, psi);
    for (int k = 0; k < p; k++) {
        phase_apply(dim, cost, angles[p + k], psi);
        general_mixer(n, d, angles[k], psi);
    }
    *E = expect(dim, cost, psi);
    for (int64_t a = 0; a < dim; a++) lam[a] = cost[a] * psi[a];
    for (int k = p - 1; k >= 0; k--) {
        general_hm(n, d, psi, hv);
        double gb = 0.0;
        for (int64_t a = 0; a < dim; a++) gb += cimag(conj(lam[a]) * hv[a]);
        grad[k] = 2.0 * gb;
        general_mixer(n, d, -angles[k], lam);
        general_mixer(n, d, -angles[k], psi);
        double gg = 0.0;
        for (int64_t a = 0; a < dim; a++) gg += cimag(conj(lam[a]) * cost[a] * psi[a]);
        grad[p + k] = 2.0 * gg;
        phase_apply(dim, cost, -angles[p + k], lam);
        phase_apply(dim, cost, -angles[p + k], psi);
    }
    free(psi); free(lam); free(hv);
    return 0;
}

/* psi <- e^{-i beta H_M} psi for the general X mixer (interleaved complex128). */
int oracle_general_mixer_apply(int n, const double *d, double beta, double *psi) {
    if (n < 1 || n > 30) return -1;
    general_mixer(n, d, beta, (cplx *)psi);
    return 0;
}

/* ------------------------------------------- single steps, for the tests */

/* psi <- e^{-i beta H_M} psi (interleaved complex128, in place). */
int oracle_mixer_apply(int kind, int n, int64_t dim, const uint64_t *states,
                       double beta, double *psi) {
    mixer_t mx;
    if (make_mixer(&mx, kind, n, dim, states)) return -1;
    cplx *t1 = NULL, *t2 = NULL;
    if (kind != ORACLE_MIXER_X) {
        t1 = malloc(sizeof(cplx) * dim); t2 = malloc(sizeof(cplx) * dim);
        if (!t1 || !t2) { free(t1); free(t2); return -2; }
    }
    mixer_apply(&mx, beta, (cplx *)psi, t1, t2);
    free(t1); free(t2);
    return 0;
}

/* out = H_M psi (interleaved complex128). */
int oracle_hm_apply(int kind, int n, int64_t dim, const uint64_t *states,
                    const double *psi, double *out) {
    mixer_t mx;
    if (make_mixer(&mx, kind, n, dim, states)) return -1;
    hm_apply(&mx, (const cplx *)psi, (cplx *)out);
    return 0;
}
