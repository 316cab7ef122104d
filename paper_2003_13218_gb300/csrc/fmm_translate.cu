// fmm_translate.cu -- M2M and L2L (Appendix B) as dense products.
//
// In level-scaled coefficients both translations are fixed linear maps per
// child octant c (w_c = child-centre offset / parent side = (+-1/4)^3):
//   L2L: Lhat_k^l(child) = sum_{n >= k, m} Lhat_n^m(parent) R_{n-k}^{m-l}(w_c) 2^{-(k+1)}
//   M2M: Mhat_n^m(parent) = sum_c sum_{k <= n, l} R_{n-k}^{m-l}(-w_c) Mhat_k^l(child_c) 2^{-k}
// so a whole level is one product with gathered columns:
//   L2L: [8 C x C] (all octants stacked) . [C x parents]   -> added to the children
//   M2M: [C x 8 C] . [8 C x parents] (the 8 children of each parent) -> parents
// The real operator matrices are built once per plan from the complex forms.
#include <math.h>

#include <type_traits>

#include "fmm_internal.cuh"

namespace fmm {

namespace {

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ inline void split_index(int j, int &n, int &m, bool &im)
{
    n = (int)sqrt((double)j);
    while (n * n > j) --n;
    while ((n + 1) * (n + 1) <= j) ++n;
    int r = j - n * n;
    m = (r + 1) / 2;
    im = (m > 0) && (r == 2 * m);
}

// unit input coefficient: C_n^m = u (u = 1 or i), C_n^{-m} = (-1)^m conj(u)
__device__ inline Cx<double> unit_pos(bool im) { return im ? Cx<double>{0, 1} : Cx<double>{1, 0}; }
__device__ inline Cx<double> unit_neg(bool im, int m)
{
    Cx<double> u = unit_pos(im);
    u.im = -u.im;
    if (m & 1) {
        u.re = -u.re;
        u.im = -u.im;
    }
    return u;
}

// L2L operators, row-major [8 nc][nc]: row c nc + j (child output j), column e (parent input)
__global__ void k_l2l_ops(int p, const double *__restrict__ Rw, double *__restrict__ A64, float *__restrict__ A32)
{
    int nc = ncoef(p);
    int64_t total = (int64_t)8 * nc * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int e = (int)(t % nc);
        int row = (int)(t / nc);
        int c = row / nc, j = row % nc;
        int k, l, n, m;
        bool oim, iim;
        split_index(j, k, l, oim);
        split_index(e, n, m, iim);
        double v = 0;
        if (n >= k) {
            const double *R = Rw + c * nc;
            Cx<double> acc = {0, 0};
            int dn = n - k;
            if (m - l >= -dn && m - l <= dn) acc = cmul(unit_pos(iim), coef(R, dn, m - l));
            if (m > 0 && -m - l >= -dn && -m - l <= dn) {
                Cx<double> t2 = cmul(unit_neg(iim, m), coef(R, dn, -m - l));
                acc.re += t2.re;
                acc.im += t2.im;
            }
            double s = ldexp(1.0, -(k + 1));
            v = s * (oim ? acc.im : acc.re);
        }
        A64[t] = v;
        A32[t] = (float)v;
        const size_t tt = (size_t)total + (size_t)e * (8 * nc) + row;  // transposed copy [nc][8 nc]
        A64[tt] = v;
        A32[tt] = (float)v;
    }
}

// M2M operators, row-major [nc][8 nc]: row j (parent output), column c nc + e (child input)
__global__ void k_m2m_ops(int p, const double *__restrict__ Rw, double *__restrict__ B64, float *__restrict__ B32)
{
    int nc = ncoef(p);
    int64_t total = (int64_t)8 * nc * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int col = (int)(t % (8 * nc));
        int j = (int)(t / (8 * nc));
        int c = col / nc, e = col % nc;
        int n, m, k, l;
        bool oim, iim;
        split_index(j, n, m, oim);
        split_index(e, k, l, iim);
        double v = 0;
        if (k <= n) {
            const double *R = Rw + c * nc;
            int dn = n - k;
            double sg = (dn & 1) ? -1.0 : 1.0;  // R(-w) = (-1)^deg R(w)
            Cx<double> acc = {0, 0};
            if (m - l >= -dn && m - l <= dn) acc = cmul(coef(R, dn, m - l), unit_pos(iim));
            if (l > 0 && m + l >= -dn && m + l <= dn) {
                Cx<double> t2 = cmul(coef(R, dn, m + l), unit_neg(iim, l));
                acc.re += t2.re;
                acc.im += t2.im;
            }
            double s = sg * ldexp(1.0, -k);
            v = s * (oim ? acc.im : acc.re);
        }
        B64[t] = v;
        B32[t] = (float)v;
        const size_t tt = (size_t)total + (size_t)col * nc + j;  // transposed copy [8 nc][nc]
        B64[tt] = v;
        B32[tt] = (float)v;
    }
}

// Dense product with gathered columns:
//   C[coff(n) + moff(m)] (+)= sum_k A[m][k] B[boff(n) + koff(k)]
// MODE 0 (M2M, parents at level l): boff = n nc, koff(k) = (k / nc) 8^l nc + k % nc,
//         coff = cell_index(l, P(n)) nc, moff(m) = m, overwrite;
// MODE 1 (L2L, children at level l): boff = cell_index(l - 1, P(n)) nc, koff(k) = k,
//         coff = n nc, moff(m) = (m / nc) 8^(l-1) nc + m % nc, accumulate.
// n runs over the parent coordinates P in x-fastest order.
template <typename T, int MODE, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_translate(int M, int64_t N, int K, int nc, int l, const T *__restrict__ A, const T *__restrict__ B,
                T *__restrict__ C)
{
    constexpr int NT = (BM / TM) * (BN / TN);
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    __shared__ int64_t bcol[BN];
    __shared__ int64_t ccol[BN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    const int np = MODE == 0 ? (1 << l) : (1 << (l - 1));  // parents per side
    const int64_t np3 = (int64_t)np * np * np;
    for (int i = tid; i < BN; i += NT) {
        int64_t n = n0 + i;
        int64_t b = 0, c = 0;
        if (n < N) {
            int px = (int)(n % np), py = (int)((n / np) % np), pz = (int)(n / ((int64_t)np * np));
            if (MODE == 0) {
                b = n * nc;
                c = cell_index(l, px, py, pz) * nc;
            } else {
                b = cell_index(l - 1, px, py, pz) * nc;
                c = n * nc;
            }
        }
        bcol[i] = b;
        ccol[i] = c;
    }
    const int tm = tid % (BM / TM), tn = tid / (BM / TM);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0;
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            int kk = e % BK, mm = e / BK;
            int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[(size_t)m * K + k] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            int kk = e % BK, nn = e / BK;
            int k = k0 + kk;
            T v = 0;
            if (n0 + nn < N && k < K) {
                int64_t ko = MODE == 0 ? (int64_t)(k / nc) * np3 * nc + (k % nc) : k;
                v = B[bcol[nn] + ko];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][tm + i * (BM / TM)];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn + j * (BN / TN)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        int nn = tn + j * (BN / TN);
        if (n0 + nn >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int m = m0 + tm + i * (BM / TM);
            if (m >= M) continue;
            if (MODE == 0) {
                C[ccol[nn] + m] = acc[i][j];
            } else {
                int64_t mo = (int64_t)(m / nc) * np3 * nc + (m % nc);
                C[ccol[nn] + mo] += acc[i][j];
            }
        }
    }
}

// FP32 register-tiled version of the same products for the fine levels.
// The operator's K runs octant by octant, each padded to KO (a multiple of 8)
// with zero columns, so a K tile never straddles two octants and no index
// needs a division.  Tiles: BM x BN outputs per block, 8 x 8 per thread
// (rows tm*4 + i and BM/2 + tm*4 + i, columns likewise, for conflict-free
// vector reads), K in steps of 8, shared memory double-buffered.
template <int MODE, int BM, int BN>
__global__ void __launch_bounds__((BM / 8) * (BN / 8), 2)
    k_translate_f32(int M, int64_t N, int nc, int KO, int l, const float *__restrict__ A, int KA,
                    const float *__restrict__ B, float *__restrict__ C)
{
    constexpr int NT = (BM / 8) * (BN / 8);
    constexpr int BK = 8;
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    __shared__ int64_t bcol[BN];
    __shared__ int64_t ccol[BN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    const int np = MODE == 0 ? (1 << l) : (1 << (l - 1));
    const int64_t np3 = (int64_t)np * np * np;
    for (int i = tid; i < BN; i += NT) {
        int64_t n = n0 + i;
        int64_t b = -1, c = 0;
        if (n < N) {
            int px = (int)(n % np), py = (int)((n / np) % np), pz = (int)(n / ((int64_t)np * np));
            if (MODE == 0) {
                b = n * nc;
                c = cell_index(l, px, py, pz) * nc;
            } else {
                b = cell_index(l - 1, px, py, pz) * nc;
                c = n * nc;
            }
        }
        bcol[i] = b;
        ccol[i] = c;
    }
    const int tiles_per_oct = KO / BK;
    const int KT = (MODE == 0 ? 8 : 1) * tiles_per_oct;
    const int64_t ostride = MODE == 0 ? np3 * nc : 0;
    __syncthreads();

    float ra[BM * BK / NT > 0 ? BM * BK / NT : 1];
    float rb[BN * BK / NT];
    auto load_tile = [&](int t) {
        const int o = t / tiles_per_oct, kb = (t % tiles_per_oct) * BK;
#pragma unroll
        for (int i = 0; i < BM * BK / NT; ++i) {
            int e = tid + i * NT;
            int mm = e / BK, kk = e % BK;
            int m = m0 + mm;
            ra[i] = m < M ? A[(size_t)m * KA + o * KO + kb + kk] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < BN * BK / NT; ++i) {
            int e = tid + i * NT;
            int nn = e / BK, kk = e % BK;
            int k = kb + kk;
            rb[i] = (bcol[nn] >= 0 && k < nc) ? B[bcol[nn] + o * ostride + k] : 0.f;
        }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
        for (int i = 0; i < BM * BK / NT; ++i) {
            int e = tid + i * NT;
            As[buf][e % BK][e / BK] = ra[i];
        }
#pragma unroll
        for (int i = 0; i < BN * BK / NT; ++i) {
            int e = tid + i * NT;
            Bs[buf][e % BK][e / BK] = rb[i];
        }
    };

    const int tm = tid % (BM / 8), tn = tid / (BM / 8);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    load_tile(0);
    store_tile(0);
    __syncthreads();
    for (int t = 0; t < KT; ++t) {
        const int buf = t & 1;
        if (t + 1 < KT) load_tile(t + 1);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][tm * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][BM / 2 + tm * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tn * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][BN / 2 + tn * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
        }
        if (t + 1 < KT) store_tile(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int nn = (j < 4 ? tn * 4 + j : BN / 2 + tn * 4 + (j - 4));
        if (n0 + nn >= N) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? tm * 4 + i : BM / 2 + tm * 4 + (i - 4));
            if (m >= M) continue;
            if (MODE == 0) {
                C[ccol[nn] + m] = acc[i][j];
            } else {
                const int c = m / nc;
                C[ccol[nn] + (int64_t)c * np3 * nc + (m - c * nc)] += acc[i][j];
            }
        }
    }
}

// operators with every octant's K padded to KO: M2M [nc][8 KO], L2L [8 nc][KO]
__global__ void k_pad_ops(int nc, int KO, const float *__restrict__ m2m, const float *__restrict__ l2l,
                          float *__restrict__ m2mP, float *__restrict__ l2lP)
{
    const int64_t n0 = (int64_t)nc * 8 * KO, n1 = (int64_t)8 * nc * KO;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n0 + n1; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n0) {
            int m = (int)(t / (8 * KO)), r = (int)(t % (8 * KO));
            int o = r / KO, kk = r % KO;
            m2mP[t] = kk < nc ? m2m[(size_t)m * 8 * nc + o * nc + kk] : 0.f;
        } else {
            int64_t u = t - n0;
            int m = (int)(u / KO), kk = (int)(u % KO);
            l2lP[u] = kk < nc ? l2l[(size_t)m * nc + kk] : 0.f;
        }
    }
}

// The same products for coarse levels (few columns): one block per
// (column, 32 outputs), the 8 warps split K, partial sums added in warp order.
// AT is the operator transposed, [K][M].
template <typename T, int MODE>
__global__ void __launch_bounds__(256)
    k_translate_small(int M, int K, int nc, int l, const T *__restrict__ AT, const T *__restrict__ B, T *__restrict__ C)
{
    __shared__ T part[8][32];
    const int64_t n = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = blockIdx.y * 32 + lane;
    const int np = MODE == 0 ? (1 << l) : (1 << (l - 1));
    const int64_t np3 = (int64_t)np * np * np;
    const int px = (int)(n % np), py = (int)((n / np) % np), pz = (int)(n / ((int64_t)np * np));
    const int64_t bcol = MODE == 0 ? n * nc : cell_index(l - 1, px, py, pz) * nc;
    const int k0 = (int)((int64_t)K * w / 8), k1 = (int)((int64_t)K * (w + 1) / 8);
    T acc = 0;
    if (m < M) {
        // M2M: K = 8 nc, so warp w covers exactly octant w
        const int64_t obase = MODE == 0 ? (int64_t)w * np3 * nc - (int64_t)w * nc : 0;
        for (int k = k0; k < k1; ++k) acc += AT[(size_t)k * M + m] * B[bcol + obase + k];
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && m < M) {
        T s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) s += part[i][lane];
        if (MODE == 0) {
            C[cell_index(l, px, py, pz) * nc + m] = s;
        } else {
            C[((int64_t)(m / nc) * np3 + n) * nc + (m % nc)] += s;
        }
    }
}

template <typename T, int MODE>
fmm_status launch_translate(Plan &P, int l, const T *A, const T *AT, const T *B, T *C)
{
    const int nc = P.nc;
    const int M = MODE == 0 ? nc : 8 * nc;
    const int K = MODE == 0 ? 8 * nc : nc;
    const int64_t N = MODE == 0 ? ((int64_t)1 << (3 * l)) : ((int64_t)1 << (3 * (l - 1)));
    if (N * ((M + 31) / 32) <= 32768) {
        dim3 grid((unsigned)N, (M + 31) / 32);
        k_translate_small<T, MODE><<<grid, 256, 0, P.stream>>>(M, K, nc, l, AT, B, C);
        FMM_LAUNCH_CHECK(P);
        return FMM_OK;
    }
    if (std::is_same<T, float>::value) {
        constexpr int BM = 64, BN = 256;
        const int KO = (nc + 7) / 8 * 8;
        const float *AP = MODE == 0 ? P.tab.m2mP32 : P.tab.l2lP32;
        const int KA = MODE == 0 ? 8 * KO : KO;
        dim3 grid(blocks_for(N, BN), (M + BM - 1) / BM);
        k_translate_f32<MODE, BM, BN><<<grid, (BM / 8) * (BN / 8), 0, P.stream>>>(
            M, N, nc, KO, l, AP, KA, (const float *)B, (float *)C);
    } else {
        constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4;
        dim3 grid(blocks_for(N, BN), (M + BM - 1) / BM);
        k_translate<T, MODE, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, P.stream>>>(M, N, K, nc, l, A, B,
                                                                                               C);
    }
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

}  // namespace

fmm_status build_translation_ops(Plan &P)
{
    const int nc = P.nc;
    const size_t n = (size_t)8 * nc * nc;
    if (!P.tab.l2l64) {  // each table followed by its transpose
        FMM_CUDA_TRY(cudaMalloc(&P.tab.l2l64, sizeof(double) * 2 * n));
        FMM_CUDA_TRY(cudaMalloc(&P.tab.l2l32, sizeof(float) * 2 * n));
        FMM_CUDA_TRY(cudaMalloc(&P.tab.m2m64, sizeof(double) * 2 * n));
        FMM_CUDA_TRY(cudaMalloc(&P.tab.m2m32, sizeof(float) * 2 * n));
    }
    k_l2l_ops<<<blocks_for(n, 256), 256, 0, P.stream>>>(P.p, P.tab.Rw64, P.tab.l2l64, P.tab.l2l32);
    FMM_LAUNCH_CHECK(P);
    k_m2m_ops<<<blocks_for(n, 256), 256, 0, P.stream>>>(P.p, P.tab.Rw64, P.tab.m2m64, P.tab.m2m32);
    FMM_LAUNCH_CHECK(P);
    const int KO = (nc + 7) / 8 * 8;
    const size_t np_ = (size_t)8 * nc * KO;
    if (!P.tab.m2mP32) {
        FMM_CUDA_TRY(cudaMalloc(&P.tab.m2mP32, sizeof(float) * np_));
        FMM_CUDA_TRY(cudaMalloc(&P.tab.l2lP32, sizeof(float) * np_));
    }
    k_pad_ops<<<blocks_for(2 * np_, 256), 256, 0, P.stream>>>(nc, KO, P.tab.m2m32, P.tab.l2l32, P.tab.m2mP32,
                                                             P.tab.l2lP32);
    FMM_LAUNCH_CHECK(P);
    return FMM_OK;
}

// M2M into level l (parents) from level l + 1
fmm_status launch_m2m(Plan &P, int l)
{
    const size_t n = (size_t)8 * P.nc * P.nc;
    if (P.precision == FMM_PREC_FP64)
        return launch_translate<double, 0>(P, l, P.tab.m2m64, P.tab.m2m64 + n, (const double *)P.M[l + 1],
                                           (double *)P.M[l]);
    return launch_translate<float, 0>(P, l, P.tab.m2m32, P.tab.m2m32 + n, (const float *)P.M[l + 1],
                                      (float *)P.M[l]);
}

// L2L from level l - 1 into level l (added to the M2L result)
fmm_status launch_l2l(Plan &P, int l)
{
    const size_t n = (size_t)8 * P.nc * P.nc;
    if (P.precision == FMM_PREC_FP64)
        return launch_translate<double, 1>(P, l, P.tab.l2l64, P.tab.l2l64 + n, (const double *)P.L[l - 1],
                                           (double *)P.L[l]);
    return launch_translate<float, 1>(P, l, P.tab.l2l32, P.tab.l2l32 + n, (const float *)P.L[l - 1],
                                      (float *)P.L[l]);
}

}  // namespace fmm
