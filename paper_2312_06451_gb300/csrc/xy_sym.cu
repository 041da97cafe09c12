// Cyclic-shift symmetry of the XY mixers on the Hamming-weight-k states.
//
// The ring mixer sum_i (X_i X_{i+1} + Y_i Y_{i+1}) and the clique mixer
// sum_{i<j} (X_i X_j + Y_i Y_j) (Sec. 2.1) both commute with the cyclic
// relabelling of the qubits, i -> i + 1 mod n.  On the weight-k states that
// relabelling permutes basis states in orbits x_0, x_1 = rot(x_0), ...,
// x_{r-1} (r divides n).  For an orbit of period r and a momentum t = 0..r-1,
// v_t = r^{-1/2} sum_j e^{-2 pi i t j / r} |x_j> is an eigenvector of the
// shift with eigenvalue e^{2 pi i m / n}, m = t n / r.  The mixer maps the span
// of all momentum-m vectors (over every orbit) into itself, and, being real,
// the real span of momenta m and n - m as well.  So in the real basis
//   m = 0:           r^{-1/2} sum_j |x_j>
//   m = n / 2:       r^{-1/2} sum_j (-1)^j |x_j>                  (r even)
//   0 < m < n / 2:   (2/r)^{1/2} sum_j cos(2 pi t j / r) |x_j>,
//                    (2/r)^{1/2} sum_j sin(2 pi t j / r) |x_j>
// the mixer is block diagonal with floor(n/2) + 1 real symmetric blocks, one
// per m, of about D / (n / 2) states each.  V diag(e^{-i b lambda}) V^T then
// costs blocks of products instead of one D x D product (the products with
// the stored eigendecomposition are what dominates the constrained mixer,
// Sec. 2.2).
//
// This file builds the orbit structure and the dense block matrices on the
// host; the per-orbit transforms run in the orbit kernel of kernels_eig.cu.
#include "qaoa.h"
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace qg {

namespace {

// Binomials up to 64 in 64-bit integers.
uint64_t binom64(int a, int b) {
    if (b < 0 || b > a) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= b; i++) r = r * (uint64_t)(a - b + i) / (uint64_t)i;
    return r;
}

// Rank of a weight-k state among all weight-k states in increasing order
// (combinatorial number system: sum over set bits c_1 < ... < c_k of C(c_i, i)).
int64_t dicke_rank(uint64_t x, const std::vector<std::vector<uint64_t>> &B) {
    int64_t r = 0;
    int i = 1;
    for (int c = 0; x; c++, x >>= 1)
        if (x & 1u) r += (int64_t)B[c][i++];
    return r;
}

}  // namespace

bool build_sym_layout(int n, int k, SymLayout &L) {
    L = SymLayout();
    if (n < 2 || n > kSymMaxN || k < 0 || k > n) return false;
    const uint64_t D64 = binom64(n, k);
    if (D64 == 0 || D64 > (uint64_t)(1 << 16)) return false;
    const int D = (int)D64;
    L.n = n;
    L.k = k;
    L.D = D;
    std::vector<std::vector<uint64_t>> B(n + 1, std::vector<uint64_t>(k + 2, 0));
    for (int a = 0; a <= n; a++)
        for (int b = 0; b <= k + 1; b++) B[a][b] = binom64(a, b);
    // the weight-k states in increasing order
    std::vector<uint64_t> st(D);
    {
        uint64_t x = k ? ((1ull << k) - 1) : 0;
        for (int a = 0; a < D; a++) {
            st[a] = x;
            if (k == 0) break;
            const uint64_t c = x & (~x + 1), r = x + c;  // next state with the same popcount
            x = (((r ^ x) >> 2) / c) | r;
        }
    }
    const uint64_t mask = n == 64 ? ~0ull : ((1ull << n) - 1);
    auto rot = [&](uint64_t x) { return ((x << 1) | (x >> (n - 1))) & mask; };
    // orbits, representative = smallest member; full-period orbits first
    std::vector<int> seen(D, 0);
    std::vector<std::vector<int>> orbits_full, orbits_short;
    for (int a = 0; a < D; a++) {
        if (seen[a]) continue;
        std::vector<int> mem;
        uint64_t x = st[a];
        do {
            const int64_t idx = dicke_rank(x, B);
            seen[idx] = 1;
            mem.push_back((int)idx);
            x = rot(x);
        } while (x != st[a]);
        (mem.size() == (size_t)n ? orbits_full : orbits_short).push_back(mem);
    }
    std::vector<std::vector<int>> orbits = orbits_full;
    orbits.insert(orbits.end(), orbits_short.begin(), orbits_short.end());
    const int nb = n / 2 + 1;  // blocks m = 0 .. floor(n/2)
    // vectors of each orbit: (block m, t, kind 0 = cos / single, 1 = sin)
    struct Vec {
        int m, t, sin;
    };
    auto orbit_vecs = [&](int r) {
        std::vector<Vec> v;
        v.push_back({0, 0, 0});
        for (int t = 1; 2 * t < r; t++) {
            v.push_back({t * n / r, t, 0});
            v.push_back({t * n / r, t, 1});
        }
        if (r % 2 == 0) v.push_back({n / 2, r / 2, 0});
        return v;
    };
    // block sizes
    std::vector<int> bdim(nb, 0);
    for (const auto &o : orbits)
        for (const Vec &v : orbit_vecs((int)o.size())) bdim[v.m]++;
    // blocks in increasing m; empty blocks dropped
    std::vector<int> bidx(nb, -1);
    for (int m = 0; m < nb; m++) {
        if (!bdim[m]) continue;
        bidx[m] = (int)L.block_dim.size();
        L.block_m.push_back(m);
        L.block_dim.push_back(bdim[m]);
    }
    const int NB = (int)L.block_dim.size();
    L.block_off.assign(NB + 1, 0);
    L.block_pos.assign(NB + 1, 0);
    for (int b = 0; b < NB; b++) {
        L.block_off[b + 1] = L.block_off[b] + L.block_dim[b];
        L.block_pos[b + 1] = L.block_pos[b] + (L.block_dim[b] + kSymPad - 1) / kSymPad * kSymPad;
    }
    L.ldp = L.block_pos[NB];
    L.pmax = 0;
    for (int b = 0; b < NB; b++) L.pmax = std::max(L.pmax, L.block_pos[b + 1] - L.block_pos[b]);
    // per-orbit tables: members, and the padded position of each vector
    std::vector<int> fill(NB, 0);
    L.orb_start.push_back(0);
    L.orbit_of.assign(D, -1);
    L.member_of.assign(D, -1);
    for (size_t o = 0; o < orbits.size(); o++) {
        const auto &mem = orbits[o];
        const int r = (int)mem.size();
        const std::vector<Vec> vs = orbit_vecs(r);
        for (int j = 0; j < r; j++) {
            L.members.push_back(mem[j]);
            L.orbit_of[mem[j]] = (int)o;
            L.member_of[mem[j]] = j;
        }
        for (const Vec &v : vs) {
            const int b = bidx[v.m];
            L.vec_pos.push_back(L.block_pos[b] + fill[b]);
            L.vec_block.push_back(b);
            L.vec_t.push_back(v.t);
            L.vec_sin.push_back(v.sin);
            fill[b]++;
        }
        L.orb_start.push_back((int)L.members.size());
    }
    L.n_orbits = (int)orbits.size();
    // basis matrices M_r[j][a] for every period r that occurs
    L.mr_off.assign(n + 1, -1);
    for (size_t o = 0; o < orbits.size(); o++) {
        const int r = (int)orbits[o].size();
        if (L.mr_off[r] >= 0) continue;
        L.mr_off[r] = (int)L.mr.size();
        const std::vector<Vec> vs = orbit_vecs(r);
        for (int j = 0; j < r; j++)
            for (int a = 0; a < r; a++) L.mr.push_back(sym_basis_value(r, vs[a].t, vs[a].sin, j));
    }
    return true;
}

// Value at member j of the real momentum vector (t, sin) of a period-r orbit.
double sym_basis_value(int r, int t, int sin_part, int j) {
    const double kPi = 3.14159265358979323846;
    if (t == 0) return 1.0 / std::sqrt((double)r);
    if (2 * t == r) return ((j & 1) ? -1.0 : 1.0) / std::sqrt((double)r);
    // the angle 2 pi t j / r reduced to a fraction of a turn first, so that
    // equal angles give bitwise equal values
    const int q = (int)(((int64_t)t * j) % r);
    const double ang = 2.0 * kPi * (double)q / (double)r;
    return std::sqrt(2.0 / (double)r) * (sin_part ? std::sin(ang) : std::cos(ang));
}

void sym_block_hamiltonians(int mixer_kind, const SymLayout &L, std::vector<double> &H) {
    // kind 0: ring (neighbours i, i+1 mod n), 1: clique (every pair i < j)
    const int n = L.n, NB = (int)L.block_dim.size();
    std::vector<size_t> hoff(NB + 1, 0);
    for (int b = 0; b < NB; b++) hoff[b + 1] = hoff[b] + (size_t)L.block_dim[b] * L.block_dim[b];
    H.assign(hoff[NB], 0.0);
    // Dicke state values and ranks
    std::vector<uint64_t> st(L.D);
    {
        uint64_t x = L.k ? ((1ull << L.k) - 1) : 0;
        for (int a = 0; a < L.D; a++) {
            st[a] = x;
            if (L.k == 0) break;
            const uint64_t c = x & (~x + 1), r = x + c;
            x = (((r ^ x) >> 2) / c) | r;
        }
    }
    std::unordered_map<uint64_t, int> rank;
    rank.reserve(L.D * 2);
    for (int a = 0; a < L.D; a++) rank[st[a]] = a;
    // block-local index of each vector: its position minus the block start
    auto local = [&](int v) { return L.vec_pos[v] - L.block_pos[L.vec_block[v]]; };
    // qubit pairs of the mixer: ring edges (i, i + 1 mod n) for every i, or
    // every pair i < j of the clique
    std::vector<std::pair<int, int>> pairs;
    if (mixer_kind == 0) {
        for (int i = 0; i < n; i++) pairs.push_back({i, (i + 1) % n});
    } else {
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) pairs.push_back({i, j});
    }
    std::vector<double> w(L.D, 0.0);
    std::vector<char> inw(L.D, 0);
    std::vector<int> touched;
    for (int o = 0; o < L.n_orbits; o++) {
        const int s0 = L.orb_start[o], r = L.orb_start[o + 1] - s0;
        for (int a = 0; a < r; a++) {
            const int va = s0 + a;  // vectors of an orbit are numbered like its members
            const int b = L.vec_block[va];
            // w = H q_a (matrix element 2 between states differing by one swap)
            touched.clear();
            for (int j = 0; j < r; j++) {
                const double q = sym_basis_value(r, L.vec_t[va], L.vec_sin[va], j);
                const uint64_t x = st[L.members[s0 + j]];
                for (const auto &pr : pairs) {
                    if (((x >> pr.first) & 1u) == ((x >> pr.second) & 1u)) continue;
                    const uint64_t y = x ^ (1ull << pr.first) ^ (1ull << pr.second);
                    const int yi = rank[y];
                    if (!inw[yi]) {
                        inw[yi] = 1;
                        touched.push_back(yi);
                    }
                    w[yi] += 2.0 * q;
                }
            }
            // project onto the vectors of block b on the orbits reached
            for (int yi : touched) {
                const double wy = w[yi];
                w[yi] = 0.0;
                inw[yi] = 0;
                const int o2 = L.orbit_of[yi], j2 = L.member_of[yi];
                const int t0 = L.orb_start[o2], r2 = L.orb_start[o2 + 1] - t0;
                for (int c = 0; c < r2; c++) {
                    const int vb = t0 + c;
                    if (L.vec_block[vb] != b) continue;
                    const double qb = sym_basis_value(r2, L.vec_t[vb], L.vec_sin[vb], j2);
                    H[hoff[b] + (size_t)local(vb) * L.block_dim[b] + local(va)] += qb * wy;
                }
            }
        }
    }
}

}  // namespace qg

extern "C" qaoa_status qaoa_xy_block_hamiltonians(int mixer, int n, int k, int *n_blocks, int64_t *block_dim,
                                                   double *H) {
    if (!n_blocks || (mixer != QAOA_XY_RING && mixer != QAOA_XY_CLIQUE)) return QAOA_ERR_INVALID;
    qg::SymLayout L;
    if (!qg::build_sym_layout(n, k, L)) return QAOA_ERR_INVALID;
    const int NB = (int)L.block_dim.size();
    if (!block_dim) {
        *n_blocks = NB;
        return QAOA_OK;
    }
    if (*n_blocks < NB) return QAOA_ERR_INVALID;
    *n_blocks = NB;
    for (int b = 0; b < NB; b++) block_dim[b] = L.block_dim[b];
    if (H) {
        std::vector<double> h;
        qg::sym_block_hamiltonians(mixer == QAOA_XY_RING ? 0 : 1, L, h);
        std::memcpy(H, h.data(), h.size() * sizeof(double));
    }
    return QAOA_OK;
}
