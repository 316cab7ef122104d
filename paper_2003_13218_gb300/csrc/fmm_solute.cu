// fmm_solute.cu -- the solute-only far-field pass of the reduced scheme for the
// solute-solvent energy (Eq. FMMcalc): Phi_u^FF at every charge, from the
// solute charges alone.
//
// With a handful of solute charges only the leaves holding them and their
// ancestors carry solute moments.  The pass therefore
//  * builds the list of active cells per level (at most NU_MAX per level),
//    P2M at the active leaves and M2M along the active ancestors;
//  * on the coarse levels 1..LD (few cells) computes the local expansion of
//    every cell in the pass's own arrays: the level-0 lattice operator, then
//    per level the M2L terms of the active cells (one block per active cell and
//    offset, every periodic image counted) summed per target with the L2L of
//    its parent, giving the full local expansion at level LD;
//  * on the finer levels evaluates M2L only onto the targets whose interaction
//    list contains an active source (at most n_il(ws) per source), kept as a
//    sorted list per level;
//  * evaluates Phi_u at every charge as the level-LD expansion plus the sparse
//    contributions found at its finer ancestors.  A local expansion is a
//    polynomial of degree p, so evaluating it at a charge directly equals
//    shifting it to the leaf with L2L first (Appendix B) up to rounding.
// When more than NU_MAX charges are solute, or the tree has no finer levels,
// the caller runs the dense pass instead.
#include <math.h>

#include <new>
#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

constexpr int NU_MAX = 64;      // solute charges handled by the sparse pass
constexpr int LD = 3;           // levels 0..LD treated densely
// targets per fine level: at most NU_MAX * n_il(ws) (mt below)
__host__ __device__ inline int max_tgt(int ws) { return NU_MAX * n_il(ws); }

struct SoluteScratch {
    int *list = nullptr;     // [NU_MAX] sorted slots of solute charges; [NU_MAX] = count
    int *cells = nullptr;    // [9][NU_MAX] active cell (linear index) per level
    int *ncells = nullptr;   // [9]
    void *MU = nullptr;      // [9][NU_MAX][nc] solute moments of the active cells
    int *flags = nullptr;    // [8^d] target marks of one level
    int *pos = nullptr;      // [8^d + 1] exclusive scan of the marks
    int *scan_tmp = nullptr;
    int *tlist = nullptr;    // [9][mt] sorted targets per fine level
    void *contrib = nullptr; // [9][mt][nc] M2L sums at those targets
    int *h_count = nullptr;  // pinned
    cudaStream_t side = nullptr;       // high-priority stream of the prologue (overlaps the full pass's M2L)
    cudaEvent_t ev_count = nullptr;    // count copied to h_count
    cudaEvent_t ev_up = nullptr;       // full upward pass done (fork)
    cudaEvent_t ev_act = nullptr;      // prologue done (join)
    cudaEvent_t ev_ready = nullptr;    // forked pass's expansions ready (Phi_u on the near stream waits)
    cudaEvent_t ev_sparse = nullptr;   // forked sparse pass done (join)
    bool count_pending = false, prologue_pending = false, sparse_forked = false;
    void *Lt = nullptr;      // [9][NU_MAX][nc] full local expansions at the active cells (FP64)
    void *Lu = nullptr;      // solute-only local expansions of every cell of levels 0..LD (class layout), T
    double *part = nullptr;  // [NU_MAX][n_il][nc] their M2L terms, one per offset
};

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ inline void cell_xyz(int64_t lin, int n, int &x, int &y, int &z)
{
    x = (int)(lin % n);
    y = (int)((lin / n) % n);
    z = (int)(lin / ((int64_t)n * n));
}

// collect the sorted slots of the solute charges (list order is irrelevant:
// the active cells are sorted afterwards); list[NU_MAX] counts all of them
__global__ void k_sol_list(int64_t N, const uint8_t *__restrict__ sol, int *__restrict__ list)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N || !sol[s]) return;
    int idx = atomicAdd(&list[NU_MAX], 1);
    if (idx < NU_MAX) list[idx] = (int)s;
}

// active cells per level: leaves of the solute charges and their ancestors,
// each list sorted by linear index and without repeats (one thread)
__global__ void k_sol_cells(int d, const int *__restrict__ list, const int *__restrict__ sleaf, int *__restrict__ cells,
                            int *__restrict__ ncells)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int n = list[NU_MAX];
    if (n > NU_MAX) n = 0;  // the dense pass runs instead: no active cells
    int cur[NU_MAX], cnt = 0;
    for (int i = 0; i < n; ++i) cur[cnt++] = sleaf[list[i]];
    for (int l = d; l >= 0; --l) {
        // sort + unique
        for (int i = 1; i < cnt; ++i) {
            int v = cur[i], j = i - 1;
            while (j >= 0 && cur[j] > v) {
                cur[j + 1] = cur[j];
                --j;
            }
            cur[j + 1] = v;
        }
        int u = 0;
        for (int i = 0; i < cnt; ++i)
            if (u == 0 || cur[i] != cur[u - 1]) cur[u++] = cur[i];
        cnt = u;
        for (int i = 0; i < cnt; ++i) cells[l * NU_MAX + i] = cur[i];
        ncells[l] = cnt;
        if (l == 0) break;
        int nl = 1 << l;
        for (int i = 0; i < cnt; ++i) {
            int x, y, z;
            cell_xyz(cur[i], nl, x, y, z);
            cur[i] = (x >> 1) + (nl >> 1) * ((y >> 1) + (nl >> 1) * (z >> 1));
        }
    }
}

// P2M of the solute charges of active leaf blockIdx.x; thread m = column m
template <typename T>
__global__ void k_sol_p2m(int p, int d, const int *__restrict__ cells, const int *__restrict__ ncells,
                          const int *__restrict__ start, const Particle<T> *__restrict__ spu, T inv_h, T *__restrict__ MU)
{
    int i = blockIdx.x;
    if (i >= ncells[d]) return;
    int m = threadIdx.x;
    if (m > p) return;
    int nc = ncoef(p);
    int leaf = cells[d * NU_MAX + i];
    T accr[P_MAX + 1], acci[P_MAX + 1];
    for (int n = 0; n <= p; ++n) accr[n] = acci[n] = 0;
    for (int s = start[leaf]; s < start[leaf + 1]; ++s) {
        Particle<T> pt = spu[s];
        if (pt.q == T(0)) continue;
        T vx = -pt.x * inv_h, vy = -pt.y * inv_h, vz = -pt.z * inv_h;
        T r2 = vx * vx + vy * vy + vz * vz;
        T dre = 1, dim = 0;
        for (int k = 1; k <= m; ++k) {
            T sc = T(-0.5) / T(k);
            T nre = sc * (vx * dre - vy * dim), nim = sc * (vx * dim + vy * dre);
            dre = nre;
            dim = nim;
        }
        T p2re = 0, p2im = 0, p1re = dre, p1im = dim;
        accr[m] += pt.q * dre;
        acci[m] += pt.q * dim;
        for (int n = m + 1; n <= p; ++n) {
            T a = T(2 * n - 1) * vz, inv = T(1) / T((n + m) * (n - m));
            T cr = (a * p1re - r2 * p2re) * inv, ci = (a * p1im - r2 * p2im) * inv;
            accr[n] += pt.q * cr;
            acci[n] += pt.q * ci;
            p2re = p1re;
            p2im = p1im;
            p1re = cr;
            p1im = ci;
        }
    }
    T *out = MU + ((size_t)d * NU_MAX + i) * nc;
    for (int n = m; n <= p; ++n) {
        out[cre(n, m)] = accr[n];
        if (m > 0) out[cim(n, m)] = acci[n];
    }
}

// M2M from the active children at level l+1 into active cell blockIdx.x of
// level l.  One warp (blockDim 32) per output (n, m) = blockIdx.y; lane = the
// child degree k, then a fixed shuffle tree.
template <typename T>
__global__ void k_sol_m2m(int p, int l, const int *__restrict__ cells, const int *__restrict__ ncells,
                          const T *__restrict__ Rw, T *__restrict__ MU)
{
    const int i = blockIdx.x;
    if (i >= ncells[l]) return;
    const int nc = ncoef(p);
    const int nl = 1 << l;
    const int kk = threadIdx.x;
    int px, py, pz;
    cell_xyz(cells[l * NU_MAX + i], nl, px, py, pz);
    const int t = blockIdx.y;
    int n = 0;
    while (tri(n + 1, 0) <= t) ++n;
    const int m = t - tri(n, 0);
    T accr = 0, acci = 0;
    if (kk <= n) {
        const int dn = n - kk;
        const T sgn = (dn & 1) ? T(-1) : T(1);
        T scale = 1;
        for (int s = 0; s < kk; ++s) scale *= T(0.5);
        for (int k = 0; k < ncells[l + 1]; ++k) {
            int cx, cy, cz;
            cell_xyz(cells[(l + 1) * NU_MAX + k], 2 * nl, cx, cy, cz);
            if ((cx >> 1) != px || (cy >> 1) != py || (cz >> 1) != pz) continue;
            const int oct = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
            const T *Mch = MU + ((size_t)(l + 1) * NU_MAX + k) * nc;
            const T *R = Rw + oct * nc;
            for (int ll = -kk; ll <= kk; ++ll) {
                const int dm = m - ll;
                if (dm < -dn || dm > dn) continue;
                Cx<T> pr = cmul(coef(R, dn, dm), coef(Mch, kk, ll));
                accr += sgn * scale * pr.re;
                acci += sgn * scale * pr.im;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        accr += __shfl_xor_sync(0xffffffffu, accr, off);
        acci += __shfl_xor_sync(0xffffffffu, acci, off);
    }
    if (kk == 0) {
        T *out = MU + ((size_t)l * NU_MAX + i) * nc;
        out[cre(n, m)] = accr;
        if (m > 0) out[cim(n, m)] = acci;
    }
}

// interaction-list test: is s = t + delta in IL(t)?  (per axis delta in
// [-2 ws - c, 2 ws + 1 - c] for target parity c, and not all |delta| <= ws)
__device__ inline bool in_il(int dx, int dy, int dz, int tx, int ty, int tz, int ws)
{
    if (dx >= -ws && dx <= ws && dy >= -ws && dy <= ws && dz >= -ws && dz <= ws) return false;
    int cx = tx & 1, cy = ty & 1, cz = tz & 1;
    return dx >= -2 * ws - cx && dx <= 2 * ws + 1 - cx && dy >= -2 * ws - cy && dy <= 2 * ws + 1 - cy &&
           dz >= -2 * ws - cz && dz <= 2 * ws + 1 - cz;
}

__device__ inline int wrap_delta(int d, int n)  // representative of d mod n in [-n/2, n/2)
{
    d %= n;
    if (d < -n / 2) d += n;
    if (d >= n / 2) d -= n;
    return d;
}

// offset of level l in the dense arrays of levels 0..LD (8^0 + ... + 8^(l-1) cells before it)
__host__ __device__ inline int64_t dense_off(int l, int nc) { return (((int64_t)1 << (3 * l)) - 1) / 7 * nc; }

// solute-only expansion of the root: the lattice operator of Eq. 12 applied to the root's solute moments
// (zero without solute charges)
template <typename T>
__global__ void k_sol_lattice(int p, const int *__restrict__ ncells, const double *__restrict__ T0,
                              const T *__restrict__ MU, T *__restrict__ Lu0)
{
    const int nc = ncoef(p);
    const bool any = ncells[0] > 0;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        double acc = 0;
        if (any)
            for (int k = 0; k < nc; ++k) acc += T0[(size_t)k * nc + j] * (double)MU[k];
        Lu0[j] = (T)acc;
    }
}

// M2L terms of the dense levels 1..LD, one block per (active source a, offset d of the window
// [-2ws-1, 2ws+1]^3): part[a][d] = T(d) . MU_a (Eq. Lcoeffdef) when the source lies in the interaction
// list of the target t = s_a - d (wrapped).  At coarse levels several offsets reach the same target (its
// periodic images): each has its own term.
template <typename T>
__global__ void k_sol_dense_m2l(int p, int l, int ws, const int *__restrict__ cells, const int *__restrict__ ncells,
                                const T *__restrict__ Top, const T *__restrict__ MU, T *__restrict__ part)
{
    const int a = blockIdx.x, b = blockIdx.y;
    if (a >= ncells[l]) return;
    const int nc = ncoef(p), n = 1 << l, h = 2 * ws + 1, side = 2 * h + 1;
    const int dx = b % side - h, dy = (b / side) % side - h, dz = b / (side * side) - h;
    int sx, sy, sz;
    cell_xyz(cells[l * NU_MAX + a], n, sx, sy, sz);
    const int tx = (sx - dx + 4 * n) & (n - 1), ty = (sy - dy + 4 * n) & (n - 1), tz = (sz - dz + 4 * n) & (n - 1);
    if (!in_il(dx, dy, dz, tx, ty, tz, ws)) return;
    const T *Tp = Top + (size_t)off_slot(dx, dy, dz, ws) * nc * nc;
    const T *Ms = MU + ((size_t)l * NU_MAX + a) * nc;
    T *out = part + ((size_t)a * side * side * side + b) * nc;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        T acc = 0;
        for (int k = 0; k < nc; ++k) acc += Tp[(size_t)k * nc + j] * Ms[k];
        out[j] = acc;
    }
}

// dense level 1 <= l <= LD of the solute-only pass, every target cell (one block each, thread j =
// coefficient j): the L2L of the parent's expansion (Eq. L2L: Lhat_k^m = 2^-(k+1) sum_{n >= k}
// Lhat_n^q R_{n-k}^{q-m}(w_c)) plus the M2L terms of k_sol_dense_m2l whose target this is, summed in
// the window's offset order (the sums do not depend on the schedule)
template <typename T>
__global__ void k_sol_dense(int p, int l, int ws, const int *__restrict__ cells, const int *__restrict__ ncells,
                            const T *__restrict__ part, const T *__restrict__ Rw, const T *__restrict__ Lpar,
                            T *__restrict__ Lout)
{
    __shared__ short hit[(4 * WS_MAX + 3) * (4 * WS_MAX + 3) * (4 * WS_MAX + 3)];
    __shared__ T sL[NC_MAX], sR[NC_MAX];
    const int nc = ncoef(p), n = 1 << l, h = 2 * ws + 1, side = 2 * h + 1, W = side * side * side;
    int tx, ty, tz;
    cell_xyz(blockIdx.x, n, tx, ty, tz);
    const int na = ncells[l];
    const int *act = cells + l * NU_MAX;
    const int oct = (tx & 1) | ((ty & 1) << 1) | ((tz & 1) << 2);
    const T *Lp = Lpar + cell_index(l - 1, tx >> 1, ty >> 1, tz >> 1) * nc;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        sL[j] = Lp[j];
        sR[j] = Rw[oct * nc + j];
    }
    for (int b = threadIdx.x; b < W; b += blockDim.x) {
        const int dx = b % side - h, dy = (b / side) % side - h, dz = b / (side * side) - h;
        int a = -1;
        if (in_il(dx, dy, dz, tx, ty, tz, ws)) {
            const int key = ((tx + dx + 4 * n) & (n - 1)) + n * (((ty + dy + 4 * n) & (n - 1)) +
                                                                 n * ((tz + dz + 4 * n) & (n - 1)));
            int lo = 0, hi = na;  // active cells are sorted and unique
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (act[mid] < key) lo = mid + 1;
                else hi = mid;
            }
            if (lo < na && act[lo] == key) a = lo;
        }
        hit[b] = (short)a;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        // output coefficient j = (k, m, real or imaginary part)
        int k = 0;
        while ((k + 1) * (k + 1) <= j) ++k;
        const int r = j - k * k;
        const int m = (r + 1) >> 1;
        const bool imag = r > 0 && (r & 1) == 0;
        T accr = 0, acci = 0;
        for (int nn = k; nn <= p; ++nn) {
            const int dn = nn - k;
            for (int q = m - dn; q <= m + dn; ++q) {
                if (q < -nn || q > nn) continue;
                Cx<T> pr = cmul(coef(sL, nn, q), coef(sR, dn, q - m));
                accr += pr.re;
                acci += pr.im;
            }
        }
        T scale = 1;
        for (int e = 0; e <= k; ++e) scale *= T(0.5);
        T acc = scale * (imag ? acci : accr);
        for (int b = 0; b < W; ++b) {
            const int a = hit[b];
            if (a >= 0) acc += part[((size_t)a * W + b) * nc + j];
        }
        Lout[cell_index(l, tx, ty, tz) * nc + j] = acc;
    }
}

// mark the targets of active source blockIdx.x at level l (threads over the candidate offsets)
__global__ void k_sol_mark(int l, int ws, const int *__restrict__ cells, const int *__restrict__ ncells,
                           int *__restrict__ flags)
{
    int i = blockIdx.x;
    if (i >= ncells[l]) return;
    const int side = off_side(ws), h = 2 * ws + 1;
    int n = 1 << l;
    int sx, sy, sz;
    cell_xyz(cells[l * NU_MAX + i], n, sx, sy, sz);
    for (int o = threadIdx.x; o < side * side * side; o += blockDim.x) {
        int dx = o % side - h, dy = (o / side) % side - h, dz = o / (side * side) - h;
        int tx = (sx - dx + 2 * n) & (n - 1), ty = (sy - dy + 2 * n) & (n - 1), tz = (sz - dz + 2 * n) & (n - 1);
        if (in_il(dx, dy, dz, tx, ty, tz, ws)) flags[tx + n * (ty + n * tz)] = 1;
    }
}

__global__ void k_sol_compact(int64_t n, int mt, const int *__restrict__ flags, const int *__restrict__ pos,
                              int *__restrict__ tlist)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c < n && flags[c]) {
        int k = pos[c];
        if (k < mt) tlist[k] = (int)c;
    }
}

// contribution of every active source to target tlist[blockIdx.x] (Eq. Lcoeffdef)
template <typename T>
__global__ void k_sol_m2l(int p, int l, int ws, const int *__restrict__ cells, const int *__restrict__ ncells,
                          const int *__restrict__ tlist, const int *__restrict__ tcount, const T *__restrict__ Top,
                          const T *__restrict__ MU, T *__restrict__ contrib)
{
    int b = blockIdx.x;
    const int mt = max_tgt(ws);
    int cnt = *tcount;
    if (cnt > mt) cnt = mt;
    if (b >= cnt) return;
    int nc = ncoef(p);
    int n = 1 << l;
    int tx, ty, tz;
    cell_xyz(tlist[b], n, tx, ty, tz);
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        T acc = 0;
        for (int s = 0; s < ncells[l]; ++s) {
            int sx, sy, sz;
            cell_xyz(cells[l * NU_MAX + s], n, sx, sy, sz);
            int dx = wrap_delta(sx - tx, n), dy = wrap_delta(sy - ty, n), dz = wrap_delta(sz - tz, n);
            if (!in_il(dx, dy, dz, tx, ty, tz, ws)) continue;
            const T *Tp = Top + (size_t)off_slot(dx, dy, dz, ws) * nc * nc + j;
            const T *Ms = MU + ((size_t)l * NU_MAX + s) * nc;
            for (int k = 0; k < nc; ++k) acc += Tp[(size_t)k * nc] * Ms[k];
        }
        contrib[((size_t)l * mt + b) * nc + j] = acc;
    }
}

// ---- full-field potential at the solute charges (the A of Eq. FMMcalc), as
// the oracle evaluates one sampled charge: M2L over the interaction list of
// each active cell from the full pass's moments (CUDA cores, no operand
// splitting), then the level-0 lattice expansion shifted down the active
// ancestors by L2L, then L2P.  The few solute charges cannot average out the
// split-operand rounding of the tensor-core M2L, so A is taken from here.

// FP64 throughout, on the solvent moments M - M_u (the field of the solvent
// at the solute charges): Lt[0][0] = T0 . (M(0) - M_u(0))
template <typename T>
__global__ void k_act_lattice(int p, const int *__restrict__ ncells, const double *__restrict__ T0,
                              const T *__restrict__ M0, const T *__restrict__ MU0, double *__restrict__ Lt)
{
    if (ncells[0] == 0) return;
    int nc = ncoef(p);
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        double acc = 0;
        for (int k = 0; k < nc; ++k) acc += T0[(size_t)k * nc + j] * ((double)M0[k] - (double)MU0[k]);
        Lt[j] = acc;
    }
}

// part[i][o] = the M2L term of the o-th interaction-list offset of active cell
// i at level l (one block per (cell, offset))
template <typename T>
__global__ void k_act_m2l(int p, int l, int ws, const int *__restrict__ cells, const int *__restrict__ ncells,
                          const double *__restrict__ Top, const T *__restrict__ M, const T *__restrict__ MU,
                          double *__restrict__ part)
{
    int i = blockIdx.x, o = blockIdx.y;
    if (i >= ncells[l]) return;
    int nc = ncoef(p);
    int n = 1 << l;
    int tx, ty, tz;
    cell_xyz(cells[l * NU_MAX + i], n, tx, ty, tz);
    int cx = tx & 1, cy = ty & 1, cz = tz & 1;
    int dx = 0, dy = 0, dz = 0, c = -1;
    for (int z = -2 * ws - cz; z <= 2 * ws + 1 - cz && c < o; ++z)
        for (int y = -2 * ws - cy; y <= 2 * ws + 1 - cy && c < o; ++y)
            for (int x = -2 * ws - cx; x <= 2 * ws + 1 - cx && c < o; ++x) {
                if (x >= -ws && x <= ws && y >= -ws && y <= ws && z >= -ws && z <= ws) continue;
                if (++c == o) {
                    dx = x;
                    dy = y;
                    dz = z;
                }
            }
    int sx = ((tx + dx) % n + n) % n, sy = ((ty + dy) % n + n) % n, sz = ((tz + dz) % n + n) % n;
    const T *Ms = M + cell_index(l, sx, sy, sz) * nc;
    // the solute part of this source, if it is an active cell
    const T *Mu = nullptr;
    int slin = sx + n * (sy + n * sz);
    for (int k = 0; k < ncells[l]; ++k)
        if (cells[l * NU_MAX + k] == slin) Mu = MU + ((size_t)l * NU_MAX + k) * nc;
    const double *Tp = Top + (size_t)off_slot(dx, dy, dz, ws) * nc * nc;
    const int nil = n_il(ws);
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
        double acc = 0;
        if (Mu)
            for (int k = 0; k < nc; ++k) acc += Tp[(size_t)k * nc + j] * ((double)Ms[k] - (double)Mu[k]);
        else
            for (int k = 0; k < nc; ++k) acc += Tp[(size_t)k * nc + j] * (double)Ms[k];
        part[((size_t)i * nil + o) * nc + j] = acc;
    }
}

// Lt[l][i] = sum of the n_il terms: one warp per (active cell, coefficient j),
// lanes take every 32nd offset, then a fixed shuffle tree (deterministic)
__global__ void k_act_sum(int p, int l, int nil, const int *__restrict__ ncells, const double *__restrict__ part,
                          double *__restrict__ Lt)
{
    const int i = blockIdx.x;
    if (i >= ncells[l]) return;
    const int nc = ncoef(p);
    const int j = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= nc) return;
    double s = 0;
    for (int o = lane; o < nil; o += 32) s += part[((size_t)i * nil + o) * nc + j];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) Lt[((size_t)l * NU_MAX + i) * nc + j] = s;
}

// Lt[l][i] += L2L of the parent's full expansion (Lt[l-1] or, at level 1, the
// lattice result L0): Lhat_k^m += sum_{n >= k} Lhat_n^q R_{n-k}^{q-m}(w_c) 2^{-(k+1)}.
// One warp (blockDim 32) per output (k, m) = blockIdx.y; lane = n - k, then a
// fixed shuffle tree.
__global__ void k_act_l2l(int p, int l, const int *__restrict__ cells, const int *__restrict__ ncells,
                          const double *__restrict__ Rw, const double *__restrict__ L0, double *__restrict__ Lt)
{
    const int i = blockIdx.x;
    if (i >= ncells[l]) return;
    const int nc = ncoef(p);
    const int nl = 1 << l;
    const int lane = threadIdx.x;
    int x, y, z;
    cell_xyz(cells[l * NU_MAX + i], nl, x, y, z);
    const double *Lp = L0;
    if (l > 1) {
        const int plin = (x >> 1) + (nl >> 1) * ((y >> 1) + (nl >> 1) * (z >> 1));
        for (int k = 0; k < ncells[l - 1]; ++k)
            if (cells[(l - 1) * NU_MAX + k] == plin) Lp = Lt + ((size_t)(l - 1) * NU_MAX + k) * nc;
    }
    const double *R = Rw + ((x & 1) | ((y & 1) << 1) | ((z & 1) << 2)) * nc;
    const int t = blockIdx.y;
    int k = 0;
    while (tri(k + 1, 0) <= t) ++k;
    const int m = t - tri(k, 0);
    double accr = 0, acci = 0;
    const int n = k + lane;
    if (n <= p) {
        const int dn = n - k;
        for (int q = -n; q <= n; ++q) {
            const int dm = q - m;
            if (dm < -dn || dm > dn) continue;
            Cx<double> pr = cmul(coef(Lp, n, q), coef(R, dn, dm));
            accr += pr.re;
            acci += pr.im;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        accr += __shfl_xor_sync(0xffffffffu, accr, off);
        acci += __shfl_xor_sync(0xffffffffu, acci, off);
    }
    if (lane == 0) {
        double scale = 1;
        for (int s = 0; s <= k; ++s) scale *= 0.5;
        double *out = Lt + ((size_t)l * NU_MAX + i) * nc;
        out[cre(k, m)] += scale * accr;
        if (m > 0) out[cim(k, m)] += scale * acci;
    }
}

template <typename T>
__device__ T l2p_value(int p, const T *__restrict__ Lc, T vx, T vy, T vz, const T *s_half = nullptr,
                       const T *s_inv = nullptr);

// at each solute charge: phi_ff = (solvent field from Lt) + phi_u (solute field
// of the solute-only pass), so that A - B = sum_u q Phi_v holds term by term
template <typename T>
__global__ void k_act_l2p(int p, int d, double inv_h, const int *__restrict__ list, const int *__restrict__ cells,
                          const int *__restrict__ ncells, const int *__restrict__ sleaf,
                          const Particle<T> *__restrict__ sp, const double *__restrict__ Lt,
                          const T *__restrict__ phi_u, T *__restrict__ phi)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    int n = list[NU_MAX];
    if (n > NU_MAX) n = NU_MAX;
    if (k >= n) return;
    int s = list[k];
    int leaf = sleaf[s];
    int i = 0;
    while (i < ncells[d] && cells[d * NU_MAX + i] != leaf) ++i;
    if (i >= ncells[d]) return;
    Particle<T> pt = sp[s];
    double v = l2p_value<double>(p, Lt + ((size_t)d * NU_MAX + i) * ncoef(p), (double)pt.x * inv_h,
                                 (double)pt.y * inv_h, (double)pt.z * inv_h) *
               inv_h;
    phi[s] = (T)(v + (double)phi_u[s]);
}

// Phi at (v) from the real-layout local coefficients Lc (scaled), v in cell units;
// s_half[m] = -1/(2m) and s_inv[n (p+1) + m] = 1/((n+m)(n-m)) when given
template <typename T>
__device__ T l2p_value(int p, const T *__restrict__ Lc, T vx, T vy, T vz, const T *s_half, const T *s_inv)
{
    T r2 = vx * vx + vy * vy + vz * vz;
    T pot = 0, dre = 1, dim = 0;
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            T sc = s_half ? s_half[m] : T(-0.5) / T(m);
            T nre = sc * (vx * dre - vy * dim), nim = sc * (vx * dim + vy * dre);
            dre = nre;
            dim = nim;
        }
        T w = m == 0 ? T(1) : T(2);
        T p2re = 0, p2im = 0, rre = dre, rim = dim;
        for (int n = m; n <= p; ++n) {
            if (n > m) {
                T a = T(2 * n - 1) * vz, inv = s_inv ? s_inv[n * (p + 1) + m] : T(1) / T((n + m) * (n - m));
                T cr = (a * rre - r2 * p2re) * inv, ci = (a * rim - r2 * p2im) * inv;
                p2re = rre;
                p2im = rim;
                rre = cr;
                rim = ci;
            }
            Cx<T> L = coef(Lc, n, m);
            pot += w * (L.re * rre - L.im * rim);
        }
    }
    return pot;
}

// Phi_u at every charge: level-LD expansion plus the sparse finer-level sums
template <typename T>
__global__ void k_sol_eval(int p, int d, int mt, int64_t N, T h_leaf, const int *__restrict__ sleaf,
                           const Particle<T> *__restrict__ sp, const T *__restrict__ Lld, const int *__restrict__ tlist,
                           const int *__restrict__ tcounts, const T *__restrict__ contrib, T *__restrict__ phi)
{
    __shared__ T s_half[P_MAX + 1];
    __shared__ T s_inv[(P_MAX + 1) * (P_MAX + 1)];
    for (int e = threadIdx.x; e < (p + 1) * (p + 1); e += blockDim.x) {
        const int n = e / (p + 1), mm = e % (p + 1);
        s_inv[e] = n > mm ? T(1) / T((n + mm) * (n - mm)) : T(0);
        if (e <= p) s_half[e] = e > 0 ? T(-0.5) / T(e) : T(0);
    }
    __syncthreads();
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int nc = ncoef(p);
    int nside = 1 << d;
    int leaf = sleaf[s];
    int x, y, z;
    cell_xyz(leaf, nside, x, y, z);
    Particle<T> pt = sp[s];
    T total = 0;
    for (int l = LD; l <= d; ++l) {
        int sh = d - l;
        int ax = x >> sh, ay = y >> sh, az = z >> sh;
        // centre of the leaf relative to the centre of its level-l ancestor, in leaf units
        T ox = T((x - (ax << sh)) + 0.5) - T(0.5) * T(1 << sh);
        T oy = T((y - (ay << sh)) + 0.5) - T(0.5) * T(1 << sh);
        T oz = T((z - (az << sh)) + 0.5) - T(0.5) * T(1 << sh);
        T inv = T(1) / (h_leaf * T(1 << sh));
        T vx = (pt.x + ox * h_leaf) * inv, vy = (pt.y + oy * h_leaf) * inv, vz = (pt.z + oz * h_leaf) * inv;
        if (l == LD) {
            total += l2p_value<T>(p, Lld + cell_index(l, ax, ay, az) * nc, vx, vy, vz, s_half, s_inv) * inv;
            continue;
        }
        int cnt = tcounts[l];
        if (cnt > mt) cnt = mt;
        int key = ax + (1 << l) * (ay + (1 << l) * az);
        const int *tl = tlist + (size_t)l * mt;
        int lo = 0, hi = cnt;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (tl[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        if (lo < cnt && tl[lo] == key)
            total += l2p_value<T>(p, contrib + ((size_t)l * mt + lo) * nc, vx, vy, vz, s_half, s_inv) * inv;
    }
    phi[s] = total;
}

// exclusive scan (one block per 4096 flags), reusing the layout of the sort's scan
__global__ void k_flag_scan_blocks(int64_t n, const int *__restrict__ in, int *__restrict__ out, int *__restrict__ sums)
{
    __shared__ int ws[32];
    int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 16;
    int v[16], local = 0;
    for (int k = 0; k < 16; ++k) {
        int64_t idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        local += v[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = local;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    int excl = x - local + (wid > 0 ? ws[wid - 1] : 0);
    for (int k = 0; k < 16; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = excl;
        excl += v[k];
    }
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = excl;
}

__global__ void k_flag_scan_sums(int nb, int *__restrict__ sums, int *__restrict__ total)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nb; ++b) {
            int t = sums[b];
            sums[b] = acc;
            acc += t;
        }
        *total = acc;
    }
}

__global__ void k_flag_scan_add(int64_t n, int *__restrict__ out, const int *__restrict__ sums)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / 4096];
}

// prologue on stream `st`: active cells, solute moments MU of the active cells
// and the FP64 local expansions Lt of the solvent field there (from the full
// pass's moments minus MU), before the rest of the pass overwrites the coarse
// moments.  Grids cover NU_MAX cells; the device count decides (no cells when
// the sparse pass does not apply).
template <typename T>
fmm_status solute_prologue_t(Plan &P, SoluteScratch &S, cudaStream_t st)
{
    const int p = P.p, d = P.d, nc = P.nc;
    const int nside = 1 << d;
    const double h = P.box / nside;
    const int nu = NU_MAX;
    const T *Rw = std::is_same<T, double>::value ? (const T *)P.tab.Rw64 : (const T *)P.tab.Rw32;
    T *MU = (T *)S.MU;
    k_sol_cells<<<1, 32, 0, st>>>(d, S.list, P.sleaf, S.cells, S.ncells);
    FMM_LAUNCH_CHECK(P);
    k_sol_p2m<T><<<nu, 32, 0, st>>>(p, d, S.cells, S.ncells, P.cell_start, (const Particle<T> *)P.sorted_u,
                                       (T)(1.0 / h), MU);
    FMM_LAUNCH_CHECK(P);
    for (int l = d - 1; l >= 0; --l) {
        k_sol_m2m<T><<<dim3(nu, (p + 1) * (p + 2) / 2), 32, 0, st>>>(p, l, S.cells, S.ncells, Rw, MU);
        FMM_LAUNCH_CHECK(P);
    }
    const int nth = ((nc + 31) / 32) * 32;
    double *Lt = (double *)S.Lt;
    k_act_lattice<T><<<1, nth, 0, st>>>(p, S.ncells, P.tab.T0, (const T *)P.M[0], MU, Lt);
    FMM_LAUNCH_CHECK(P);
    for (int l = 1; l <= d; ++l) {
        k_act_m2l<T><<<dim3(nu, n_il(P.ws)), nth, 0, st>>>(p, l, P.ws, S.cells, S.ncells, P.tab.Top64,
                                                            (const T *)P.M[l], MU, S.part);
        FMM_LAUNCH_CHECK(P);
        k_act_sum<<<dim3(nu, (nc + 7) / 8), 256, 0, st>>>(p, l, n_il(P.ws), S.ncells, S.part, Lt);
        FMM_LAUNCH_CHECK(P);
        k_act_l2l<<<dim3(nu, (p + 1) * (p + 2) / 2), 32, 0, st>>>(p, l, S.cells, S.ncells, P.tab.Rw64, Lt, Lt);
        FMM_LAUNCH_CHECK(P);
    }
    return FMM_OK;
}

// the rest of the pass (it reads only the prologue's active cells and moments): the dense coarse levels
// into the pass's own arrays and the target lists and M2L sums of the sparse finer levels
template <typename T>
fmm_status solute_sparse_t(Plan &P, SoluteScratch &S, int nu)
{
    const int p = P.p, d = P.d, nc = P.nc;
    const T *Top = std::is_same<T, double>::value ? (const T *)P.tab.Top64 : (const T *)P.tab.Top32;
    const T *Rw = std::is_same<T, double>::value ? (const T *)P.tab.Rw64 : (const T *)P.tab.Rw32;
    T *MU = (T *)S.MU;
    T *Lu = (T *)S.Lu;
    const int nth = ((nc + 31) / 32) * 32;
    // dense coarse levels 0..LD
    k_sol_lattice<T><<<1, nth, 0, P.stream>>>(p, S.ncells, P.tab.T0, MU, Lu);
    FMM_LAUNCH_CHECK(P);
    // the M2L terms of one dense level at a time in the (unused) level 0..LD part of the sparse sums
    T *part = (T *)S.contrib;
    const int win = off_side(P.ws) * off_side(P.ws) * off_side(P.ws);
    for (int l = 1; l <= LD; ++l) {
        k_sol_dense_m2l<T><<<dim3(nu, win), nth, 0, P.stream>>>(p, l, P.ws, S.cells, S.ncells, Top, MU, part);
        FMM_LAUNCH_CHECK(P);
        k_sol_dense<T><<<1u << (3 * l), nth, 0, P.stream>>>(p, l, P.ws, S.cells, S.ncells, part, Rw,
                                                              Lu + dense_off(l - 1, nc), Lu + dense_off(l, nc));
        FMM_LAUNCH_CHECK(P);
    }
    // sparse finer levels
    for (int l = LD + 1; l <= d; ++l) {
        int64_t n = (int64_t)1 << (3 * l);
        FMM_CUDA_TRY(cudaMemsetAsync(S.flags, 0, sizeof(int) * n, P.stream));
        k_sol_mark<<<nu, 256, 0, P.stream>>>(l, P.ws, S.cells, S.ncells, S.flags);
        FMM_LAUNCH_CHECK(P);
        int nb = (int)((n + 4095) / 4096);
        k_flag_scan_blocks<<<nb, 256, 0, P.stream>>>(n, S.flags, S.pos, S.scan_tmp);
        FMM_LAUNCH_CHECK(P);
        k_flag_scan_sums<<<1, 32, 0, P.stream>>>(nb, S.scan_tmp, S.ncells + 16 + l);
        FMM_LAUNCH_CHECK(P);
        k_flag_scan_add<<<blocks_for(n, 256), 256, 0, P.stream>>>(n, S.pos, S.scan_tmp);
        FMM_LAUNCH_CHECK(P);
        k_sol_compact<<<blocks_for(n, 256), 256, 0, P.stream>>>(n, max_tgt(P.ws), S.flags, S.pos,
                                                                 S.tlist + (size_t)l * max_tgt(P.ws));
        FMM_LAUNCH_CHECK(P);
        k_sol_m2l<T><<<nu * n_il(P.ws), ((nc + 31) / 32) * 32, 0, P.stream>>>(p, l, P.ws, S.cells, S.ncells,
                                                                       S.tlist + (size_t)l * max_tgt(P.ws),
                                                                       S.ncells + 16 + l, Top, MU, (T *)S.contrib);
        FMM_LAUNCH_CHECK(P);
    }
    return FMM_OK;
}

// Phi_u at every charge: the level-LD expansion plus the sparse finer-level sums
template <typename T>
fmm_status solute_eval_t(Plan &P, SoluteScratch &S)
{
    const double h = P.box / (1 << P.d);
    k_sol_eval<T><<<blocks_for(P.N, 128), 128, 0, P.stream>>>(P.p, P.d, max_tgt(P.ws), P.N, (T)h, P.sleaf,
                                                              (const Particle<T> *)P.sorted,
                                                              (const T *)S.Lu + dense_off(LD, P.nc), S.tlist,
                                                              S.ncells + 16, (const T *)S.contrib, (T *)P.phi_u);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

// full-field potential at the solute charges (solvent field + solute field) into phi_ff, after the full
// pass's L2P has written phi_ff
template <typename T>
fmm_status solute_act_l2p_t(Plan &P, SoluteScratch &S)
{
    const double h = P.box / (1 << P.d);
    k_act_l2p<T><<<1, NU_MAX, 0, P.stream>>>(P.p, P.d, 1.0 / h, S.list, S.cells, S.ncells, P.sleaf,
                                             (const Particle<T> *)P.sorted, (const double *)S.Lt,
                                             (const T *)P.phi_u, (T *)P.phi_ff);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

}  // namespace

fmm_status solute_prepare(Plan &P)
{
    solute_free(P);
    if (P.d <= LD) return FMM_OK;
    SoluteScratch *S = new (std::nothrow) SoluteScratch();
    if (!S) return FMM_ERR_OOM;
    P.sol = S;
    int64_t nleaf = (int64_t)1 << (3 * P.d);
    FMM_CUDA_TRY(cudaMalloc(&S->list, sizeof(int) * (NU_MAX + 4)));
    FMM_CUDA_TRY(cudaMalloc(&S->cells, sizeof(int) * 9 * NU_MAX));
    FMM_CUDA_TRY(cudaMalloc(&S->ncells, sizeof(int) * 32));
    FMM_CUDA_TRY(cudaMalloc(&S->MU, sizeof(double) * 9 * NU_MAX * P.nc));
    FMM_CUDA_TRY(cudaMalloc(&S->flags, sizeof(int) * nleaf));
    FMM_CUDA_TRY(cudaMalloc(&S->pos, sizeof(int) * (nleaf + 1)));
    FMM_CUDA_TRY(cudaMalloc(&S->scan_tmp, sizeof(int) * (nleaf / 4096 + 2)));
    FMM_CUDA_TRY(cudaMalloc(&S->tlist, sizeof(int) * 9 * max_tgt(P.ws)));
    FMM_CUDA_TRY(cudaMalloc(&S->contrib, sizeof(double) * (size_t)(P.d + 1) * max_tgt(P.ws) * P.nc));
    FMM_CUDA_TRY(cudaMallocHost((void **)&S->h_count, sizeof(int)));
    int lo = 0, hi = 0;
    FMM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    FMM_CUDA_TRY(cudaStreamCreateWithPriority(&S->side, cudaStreamNonBlocking, hi));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_count, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_up, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_act, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_ready, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaEventCreateWithFlags(&S->ev_sparse, cudaEventDisableTiming));
    FMM_CUDA_TRY(cudaMalloc(&S->Lt, sizeof(double) * 9 * NU_MAX * P.nc));
    FMM_CUDA_TRY(cudaMalloc(&S->Lu, sizeof(double) * dense_off(LD + 1, P.nc)));
    FMM_CUDA_TRY(cudaMalloc(&S->part, sizeof(double) * NU_MAX * n_il(P.ws) * P.nc));
    return FMM_OK;
}

void solute_free(Plan &P)
{
    SoluteScratch *S = (SoluteScratch *)P.sol;
    if (!S) return;
    cudaFree(S->list);
    cudaFree(S->cells);
    cudaFree(S->ncells);
    cudaFree(S->MU);
    cudaFree(S->flags);
    cudaFree(S->pos);
    cudaFree(S->scan_tmp);
    cudaFree(S->tlist);
    cudaFree(S->contrib);
    cudaFree(S->Lt);
    cudaFree(S->Lu);
    cudaFree(S->part);
    if (S->h_count) cudaFreeHost(S->h_count);
    if (S->side) {
        cudaStreamSynchronize(S->side);
        cudaStreamDestroy(S->side);
    }
    if (S->ev_count) cudaEventDestroy(S->ev_count);
    if (S->ev_up) cudaEventDestroy(S->ev_up);
    if (S->ev_act) cudaEventDestroy(S->ev_act);
    if (S->ev_ready) cudaEventDestroy(S->ev_ready);
    if (S->ev_sparse) cudaEventDestroy(S->ev_sparse);
    delete S;
    P.sol = nullptr;
}

int solute_count_host(const Plan &P)
{
    const SoluteScratch *S = (const SoluteScratch *)P.sol;
    return S ? *S->h_count : -1;
}

fmm_status solute_count(Plan &P)
{
    SoluteScratch *S = (SoluteScratch *)P.sol;
    if (!S) return FMM_OK;
    S->sparse_forked = false;  // a new call (a failed one may have left it set)
    FMM_CUDA_TRY(cudaMemsetAsync(S->list + NU_MAX, 0, sizeof(int), P.stream));
    k_sol_list<<<blocks_for(P.N, 256), 256, 0, P.stream>>>(P.N, P.sorted_sol, S->list);
    FMM_LAUNCH_CHECK(P);
    FMM_CUDA_TRY(cudaMemcpyAsync(S->h_count, S->list + NU_MAX, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    FMM_CUDA_TRY(cudaEventRecord(S->ev_count, P.stream));
    S->count_pending = true;
    return FMM_OK;
}

fmm_status solute_prologue(Plan &P)
{
    SoluteScratch *S = (SoluteScratch *)P.sol;
    if (!S) return FMM_OK;
    if (!S->count_pending) {
        fmm_status s = solute_count(P);
        if (s != FMM_OK) return s;
    }
    FMM_CUDA_TRY(cudaEventRecord(S->ev_up, P.stream));
    FMM_CUDA_TRY(cudaStreamWaitEvent(S->side, S->ev_up, 0));
    fmm_status s = P.precision == FMM_PREC_FP64 ? solute_prologue_t<double>(P, *S, S->side)
                                                : solute_prologue_t<float>(P, *S, S->side);
    FMM_CUDA_TRY(cudaEventRecord(S->ev_act, S->side));
    S->prologue_pending = true;
    return s;
}

fmm_status solute_sparse_fork(Plan &P)
{
    SoluteScratch *S = (SoluteScratch *)P.sol;
    if (!S || !P.overlap || !S->prologue_pending || S->sparse_forked) return FMM_OK;
    int nu = NU_MAX;  // unknown count: grids for the largest, the device count decides
    if (P.known_count >= 0) {
        if (P.known_count == 0 || P.known_count > NU_MAX) return FMM_OK;  // nothing to overlap
        nu = P.known_count;
    }
    // behind the prologue on the side stream; Phi_u at every charge (a full-size launch) on the near
    // stream, where it fills idle SMs instead of taking them from the far field
    cudaStream_t main_stream = P.stream;
    P.stream = S->side;
    fmm_status s = P.precision == FMM_PREC_FP64 ? solute_sparse_t<double>(P, *S, nu) : solute_sparse_t<float>(P, *S, nu);
    if (s == FMM_OK && P.near_forked) {
        if (cudaEventRecord(S->ev_ready, S->side) != cudaSuccess || cudaStreamWaitEvent(P.near, S->ev_ready, 0) != cudaSuccess)
            s = FMM_ERR_CUDA;
        P.stream = P.near;
    }
    if (s == FMM_OK) s = P.precision == FMM_PREC_FP64 ? solute_eval_t<double>(P, *S) : solute_eval_t<float>(P, *S);
    P.stream = main_stream;
    if (s != FMM_OK) return s;
    FMM_CUDA_TRY(cudaEventRecord(S->ev_sparse, S->side));
    S->sparse_forked = true;
    return FMM_OK;
}

// Phi_u into P.phi_u by the sparse pass; *done = false asks for the dense pass
fmm_status launch_solute_pass(Plan &P, bool *done)
{
    *done = false;
    SoluteScratch *S = (SoluteScratch *)P.sol;
    if (!S) return FMM_OK;
    if (S->sparse_forked) {
        // forked after the prologue (Phi_u on the near stream, joined before this call): join the side
        // stream; the dense pass overwrites the (empty) result when the count is above NU_MAX
        if (P.known_count < 0) FMM_CUDA_TRY(cudaEventSynchronize(S->ev_count));
        FMM_CUDA_TRY(cudaStreamWaitEvent(P.stream, S->ev_sparse, 0));
        S->count_pending = S->prologue_pending = S->sparse_forked = false;
        int n = P.known_count >= 0 ? P.known_count : *S->h_count;
        if (n > NU_MAX) return FMM_OK;
        if (n == 0) {
            size_t bytes = (P.precision == FMM_PREC_FP64 ? sizeof(double) : sizeof(float)) * P.N;
            FMM_CUDA_TRY(cudaMemsetAsync(P.phi_u, 0, bytes, P.stream));
            *done = true;
            return FMM_OK;
        }
        fmm_status s = P.precision == FMM_PREC_FP64 ? solute_act_l2p_t<double>(P, *S) : solute_act_l2p_t<float>(P, *S);
        if (s == FMM_OK) *done = true;
        return s;
    }
    if (!S->prologue_pending) {
        fmm_status s = solute_prologue(P);
        if (s != FMM_OK) return s;
    }
    // the count was copied right after the sort (or the caller knows it); the join orders the
    // prologue before the rest
    if (P.known_count < 0) FMM_CUDA_TRY(cudaEventSynchronize(S->ev_count));
    FMM_CUDA_TRY(cudaStreamWaitEvent(P.stream, S->ev_act, 0));
    S->count_pending = S->prologue_pending = false;
    int n = P.known_count >= 0 ? P.known_count : *S->h_count;
    if (n > NU_MAX) return FMM_OK;
    if (n == 0) {
        size_t bytes = (P.precision == FMM_PREC_FP64 ? sizeof(double) : sizeof(float)) * P.N;
        FMM_CUDA_TRY(cudaMemsetAsync(P.phi_u, 0, bytes, P.stream));
        *done = true;
        return FMM_OK;
    }
    fmm_status s = P.precision == FMM_PREC_FP64 ? solute_sparse_t<double>(P, *S, n) : solute_sparse_t<float>(P, *S, n);
    if (s == FMM_OK) s = P.precision == FMM_PREC_FP64 ? solute_eval_t<double>(P, *S) : solute_eval_t<float>(P, *S);
    if (s == FMM_OK) s = P.precision == FMM_PREC_FP64 ? solute_act_l2p_t<double>(P, *S) : solute_act_l2p_t<float>(P, *S);
    if (s == FMM_OK) *done = true;
    return s;
}

}  // namespace fmm
