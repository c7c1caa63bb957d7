// eri_tables.cu -- device copies of the generated Rys/Boys tables and the component
// diagnostics eri_boys_device / eri_rys_device (same device code as the ERI kernels).
#include <mutex>
#include <vector>

#include "eri_device.cuh"
#include "eri_internal.h"
#include "eri_tables.inc"

static_assert(RYS_NMAX == eri::kRysNmax, "table order mismatch");
static_assert(RYS_DEG == eri::kRysDeg, "table degree mismatch");
static_assert(RYS_TAIL == eri::kRysTail, "table tail mismatch");
static_assert(RYS_TAIL_LEN * (RYS_DEG + 1) == RYS_POLY_LEN * (RYS_DEG + 1 - RYS_TAIL), "tail size");
static_assert(BOYS_MMAX == eri::kBoysMmax && BOYS_TAYLOR == eri::kBoysTaylor &&
                  BOYS_MCOLS == eri::kBoysCols && BOYS_NGRID == eri::kBoysNgrid,
              "Boys grid mismatch");
static_assert(BOYS_T01_LEN == 2 * BOYS_TAYLOR * BOYS_NGRID, "F0/F1 Taylor table size");

namespace eri {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_tables_mutex;
bool g_tables_ready[kMaxDevices];
Tables g_tables[kMaxDevices];
}  // namespace

// FP32 copies for the mixed-precision setup: coefficients kRysTailMixed..kRysDeg of every
// root/weight piece, and the F_0/F_1 Taylor table (round to nearest).
void mixed_table_copies(std::vector<float> &tail_m, std::vector<float> &t01_f) {
    const int pieces = RYS_POLY_LEN / (RYS_DEG + 1);
    const int keep = RYS_DEG + 1 - kRysTailMixed;
    tail_m.resize((size_t)pieces * keep);
    for (int f = 0; f < pieces; ++f)
        for (int j = 0; j < keep; ++j)
            tail_m[(size_t)f * keep + j] = (float)rys_poly_h[(size_t)f * (RYS_DEG + 1) + kRysTailMixed + j];
    t01_f.resize(BOYS_T01_LEN);
    for (int i = 0; i < BOYS_T01_LEN; ++i) t01_f[i] = (float)boys_t01_h[i];
}

// Uploads the tables to the current device once; returns the device addresses.
cudaError_t tables_for_current_device(Tables *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_tables_mutex);
    if (!g_tables_ready[dev]) {
        Tables t{};
        double *buf = nullptr;
        std::vector<float> tail_m, t01_f;
        mixed_table_copies(tail_m, t01_f);
        size_t n = (size_t)RYS_POLY_LEN + 2 * (size_t)RYS_HERM_LEN + (size_t)BOYS_GRID_LEN +
                   (size_t)BOYS_T01_LEN + ((size_t)RYS_TAIL_LEN + 1) / 2 + (tail_m.size() + 1) / 2 +
                   (t01_f.size() + 1) / 2;
        e = cudaMalloc(&buf, n * sizeof(double));
        if (e != cudaSuccess) return e;
        double *p = buf;
        e = cudaMemcpy(p, rys_poly_h, sizeof(rys_poly_h), cudaMemcpyHostToDevice);
        t.rys_poly = p;
        p += RYS_POLY_LEN;
        if (e == cudaSuccess) e = cudaMemcpy(p, rys_herm_x2_h, sizeof(rys_herm_x2_h), cudaMemcpyHostToDevice);
        t.herm_x2 = p;
        p += RYS_HERM_LEN;
        if (e == cudaSuccess) e = cudaMemcpy(p, rys_herm_w_h, sizeof(rys_herm_w_h), cudaMemcpyHostToDevice);
        t.herm_w = p;
        p += RYS_HERM_LEN;
        if (e == cudaSuccess) e = cudaMemcpy(p, boys_grid_h, sizeof(boys_grid_h), cudaMemcpyHostToDevice);
        t.boys_grid = p;
        p += BOYS_GRID_LEN;
        if (e == cudaSuccess) e = cudaMemcpy(p, boys_t01_h, sizeof(boys_t01_h), cudaMemcpyHostToDevice);
        t.boys_t01 = p;
        p += BOYS_T01_LEN;
        if (e == cudaSuccess) e = cudaMemcpy(p, rys_tail_f_h, sizeof(rys_tail_f_h), cudaMemcpyHostToDevice);
        t.rys_tail = reinterpret_cast<const float *>(p);
        p += ((size_t)RYS_TAIL_LEN + 1) / 2;
        if (e == cudaSuccess)
            e = cudaMemcpy(p, tail_m.data(), tail_m.size() * sizeof(float), cudaMemcpyHostToDevice);
        t.rys_tail_m = reinterpret_cast<const float *>(p);
        p += (tail_m.size() + 1) / 2;
        if (e == cudaSuccess)
            e = cudaMemcpy(p, t01_f.data(), t01_f.size() * sizeof(float), cudaMemcpyHostToDevice);
        t.boys_t01_f = reinterpret_cast<const float *>(p);
        if (e != cudaSuccess) {
            cudaFree(buf);
            return e;
        }
        for (int i = 0; i <= RYS_NMAX; ++i) {
            t.tasym[i] = rys_tasym_h[i];
            t.offset[i] = rys_offset_h[i];
        }
        for (int i = 0; i <= RYS_NMAX + 1; ++i) t.herm_off[i] = rys_herm_offset_h[i];
        g_tables[dev] = t;
        g_tables_ready[dev] = true;
    }
    *out = g_tables[dev];
    return cudaSuccess;
}

__global__ void boys_kernel(Tables tb, int mmax, const double *__restrict__ T, long long n,
                            double *__restrict__ F) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double f[kBoysMmax + 1];
    boys_eval(mmax, T[i], tb.boys_grid, f);
    for (int m = 0; m <= mmax; ++m) F[i * (mmax + 1) + m] = f[m];
}

template <bool MIXED>
__global__ void rys_kernel(Tables tb, int nroots, const double *__restrict__ T, long long n,
                           double *__restrict__ X, double *__restrict__ W) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * nroots) return;
    long long k = i / nroots;
    int mu = (int)(i % nroots);
    double x, w;
    rys_root<MIXED>(tb, nroots, mu, T[k], x, w);
    X[i] = x;
    W[i] = w;
}

__global__ void convert_kernel(const double *in, long long n, float *f, double *back) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = f64_to_f32(in[i]);
    f[i] = v;
    back[i] = f32_to_f64(v);
}

// FMA throughput probe: kFmaChains independent chains of 16 * `iters` fused multiply-adds per
// thread (operands depend on the thread, the result is stored, so nothing folds away).
constexpr int kFmaChains = 16;
template <typename T>
__global__ void fma_probe_kernel(int iters, T b, T c, T *__restrict__ sink) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = (T)(tid % 1024) * (T)1e-3 + (T)k;
#pragma unroll 1
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], b, c);
    T s = 0;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    sink[tid] = s;
}

}  // namespace eri

using namespace eri;

extern "C" eri_status_t eri_fma_probe(int32_t precision, int64_t n_threads, int32_t iters, void *d_sink,
                                      void *stream) {
    if ((precision != ERI_FP64 && precision != ERI_MIXED) || n_threads < 256 || n_threads % 256 ||
        n_threads / 256 > 0x7fffffffLL || iters < 1 || !d_sink)
        return ERI_E_INVALID;
    const unsigned blocks = (unsigned)(n_threads / 256);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == ERI_FP64)
        fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7, static_cast<double *>(d_sink));
    else
        fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.9999f, 1e-4f, static_cast<float *>(d_sink));
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}

extern "C" eri_status_t eri_boys_device(int32_t mmax, const double *d_T, int64_t n, double *d_F,
                                        void *stream) {
    if (mmax < 0 || mmax > kBoysMmax || n < 0 || (n > 0 && (!d_T || !d_F))) return ERI_E_INVALID;
    if (n == 0) return ERI_OK;
    Tables tb;
    if (tables_for_current_device(&tb) != cudaSuccess) return ERI_E_CUDA;
    long long blocks = (n + 255) / 256;
    boys_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(tb, mmax, d_T, n, d_F);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}

namespace {
eri_status_t rys_device(bool mixed, int32_t nroots, const double *d_T, int64_t n, double *d_x,
                        double *d_w, void *stream) {
    if (nroots < 1 || nroots > kRysNmax || n < 0 || (n > 0 && (!d_T || !d_x || !d_w)))
        return ERI_E_INVALID;
    if (n == 0) return ERI_OK;
    Tables tb;
    if (tables_for_current_device(&tb) != cudaSuccess) return ERI_E_CUDA;
    long long total = n * nroots;
    long long blocks = (total + 255) / 256;
    if (mixed)
        rys_kernel<true><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(tb, nroots, d_T, n, d_x, d_w);
    else
        rys_kernel<false><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(tb, nroots, d_T, n, d_x, d_w);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}
}  // namespace

extern "C" eri_status_t eri_rys_device(int32_t nroots, const double *d_T, int64_t n, double *d_x,
                                       double *d_w, void *stream) {
    return rys_device(false, nroots, d_T, n, d_x, d_w, stream);
}

extern "C" eri_status_t eri_rys_device_mixed(int32_t nroots, const double *d_T, int64_t n, double *d_x,
                                             double *d_w, void *stream) {
    return rys_device(true, nroots, d_T, n, d_x, d_w, stream);
}


extern "C" eri_status_t eri_convert_device(const double *d_in, int64_t n, float *d_f, double *d_back,
                                           void *stream) {
    if (n < 0 || (n > 0 && (!d_in || !d_f || !d_back))) return ERI_E_INVALID;
    if (n == 0) return ERI_OK;
    convert_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_in, n, d_f, d_back);
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}
