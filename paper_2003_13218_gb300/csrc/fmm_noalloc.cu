// fmm_noalloc.cu -- an entry point that allocates no memory at all.
//
// fmm_background_terms_noalloc computes the background-charge terms of the
// energy (charged-system, quadrupole-surface and dipole-surface terms) and the
// moments they are built from, exactly as fmm_energy reports them, but without
// a plan and without any device allocation.  It is meant for callers that
// cannot call cudaMalloc: a host application or plug-in whose device memory is
// entirely owned by another allocator or a fixed memory budget (a second
// allocator would fragment or exceed it), and latency-sensitive loops that
// cannot afford the device-wide synchronisation cudaMalloc/cudaFree may imply.
// Non-finite charges or coordinates are not filtered: they make the affected
// outputs non-finite, which is how the caller sees them (nothing here returns
// a device-side status).
//
// Its only scratch -- one row of compensated partial sums per block of 4096
// charges -- lives in the file-scope device array below (80 KiB, held by every
// GPU that loads this library until the process exits).  Host code cannot use
// the array's name as a device address, so the address is looked up once per
// device with cudaGetSymbolAddress on the first call made while that device is
// current.  Each call writes every partial-sum row it later reads, so nothing
// has to be cleared between calls; calls that overlap on the GPU (other
// streams, other host threads) share the array and race.
#include <math.h>
#include <mutex>

#include "fmm_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CHUNK = 4096;                  // charges per block
constexpr int64_t NA_MAX_N = (int64_t)1 << 22;  // 4,194,304 charges
constexpr int NA_MAX_BLOCKS = (int)(NA_MAX_N / NA_CHUNK);
constexpr int NA_Q = 5;                         // Q, mu_x, mu_y, mu_z, S2
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_partials[NA_MAX_BLOCKS * NA_Q * 2];

struct Comp {  // Neumaier compensated sum
    double s, c;
    __device__ void add(double x)
    {
        double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
};

// one block per chunk of NA_CHUNK charges: compensated sums of q, q r, q r^2
// over coordinates wrapped into [0, b) (the same IEEE arithmetic as the
// plan's leaf assignment), written to row blockIdx.x of the scratch array
__global__ void k_na_partial(int64_t N, const double *__restrict__ pos, const double *__restrict__ q, double box,
                             double *__restrict__ partials)
{
    __shared__ double sh[NA_THREADS][2];
    Comp acc[NA_Q];
    for (int k = 0; k < NA_Q; ++k) acc[k] = {0.0, 0.0};
    const int64_t begin = (int64_t)blockIdx.x * NA_CHUNK;
    const int64_t end = begin + NA_CHUNK < N ? begin + NA_CHUNK : N;
    for (int64_t i = begin + threadIdx.x; i < end; i += NA_THREADS) {
        const double qi = q[i];  // NaN / Inf flow into the sums
        double w[3];
        for (int a = 0; a < 3; ++a) {
            const double x = pos[3 * i + a];  // NaN or Inf: floor and the subtraction yield NaN
            double f = floor(__ddiv_rn(x, box));
            double v = __dsub_rn(x, __dmul_rn(box, f));
            if (v >= box) v = __dsub_rn(v, box);
            if (v < 0.0) v = 0.0;
            w[a] = v;
        }
        acc[0].add(qi);
        acc[1].add(qi * w[0]);
        acc[2].add(qi * w[1]);
        acc[3].add(qi * w[2]);
        acc[4].add(qi * (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]));
    }
    for (int k = 0; k < NA_Q; ++k) {
        sh[threadIdx.x][0] = acc[k].s;
        sh[threadIdx.x][1] = acc[k].c;
        __syncthreads();
        for (int o = NA_THREADS / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) {
                Comp x{sh[threadIdx.x][0], sh[threadIdx.x][1]};
                x.add(sh[threadIdx.x + o][0]);
                x.add(sh[threadIdx.x + o][1]);
                sh[threadIdx.x][0] = x.s;
                sh[threadIdx.x][1] = x.c;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            partials[(blockIdx.x * NA_Q + k) * 2] = sh[0][0];
            partials[(blockIdx.x * NA_Q + k) * 2 + 1] = sh[0][1];
        }
        __syncthreads();
    }
}

// sums the rows in block order, then the three terms of the energy:
// out = {Q, mu_x, mu_y, mu_z, S2, charged, quad_surface, dipole_surface}
__global__ void k_na_final(int nblocks, const double *__restrict__ partials, double box, double kappa,
                           double *__restrict__ out)
{
    __shared__ double m[NA_Q];
    const int k = threadIdx.x;
    if (k < NA_Q) {
        Comp c{0.0, 0.0};
        for (int b = 0; b < nblocks; ++b) {
            c.add(partials[(b * NA_Q + k) * 2]);
            c.add(partials[(b * NA_Q + k) * 2 + 1]);
        }
        m[k] = c.s + c.c;
        out[k] = m[k];
    }
    __syncthreads();
    if (k == 0) {
        const double PI = 3.14159265358979323846;
        const double V = box * box * box;
        out[5] = -PI / (2.0 * V * kappa * kappa) * m[0] * m[0];
        out[6] = 2.0 * PI / (3.0 * V) * m[0] * m[4];
        out[7] = -2.0 * PI / (3.0 * V) * (m[1] * m[1] + m[2] * m[2] + m[3] * m[3]);
    }
}

std::mutex g_lookup_lock;
double *g_scratch_ptr[NA_MAX_DEVICES] = {};

// device address of g_partials on the current device (looked up once per device)
fmm_status scratch_for_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return FMM_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lookup_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return FMM_ERR_CUDA;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return FMM_OK;
}

}  // namespace

extern "C" fmm_status fmm_background_terms_noalloc(const double *pos, const double *q, int64_t N, double box,
                                                   double kappa, double *out, void *stream)
{
    if (!pos || !q || !out || N < 1 || !(box > 0.0) || !isfinite(box) || !isfinite(kappa)) return FMM_ERR_INVALID_ARG;
    if (N > NA_MAX_N) return FMM_ERR_INVALID_ARG;  // the static scratch holds NA_MAX_N / 4096 rows
    double *scratch = nullptr;
    fmm_status s = scratch_for_current_device(&scratch);
    if (s != FMM_OK) return s;
    if (!(kappa > 0.0)) kappa = 2.0 / box;
    const int nblocks = (int)((N + NA_CHUNK - 1) / NA_CHUNK);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_partial<<<nblocks, NA_THREADS, 0, st>>>(N, pos, q, box, scratch);
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    k_na_final<<<1, 32, 0, st>>>(nblocks, scratch, box, kappa, out);
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    return FMM_OK;
}
