// eri_screen.cu -- quartet lists built on the device: the 8-fold unique quartets of a shell set
// (Sec. II-B) and Schwarz screening, |(ij|kl)| <= sqrt((ij|ij)) sqrt((kl|kl)) = Q_ij Q_kl.
//
// Unordered shell pairs are numbered P(i, j) = i (i + 1) / 2 + j for i >= j.  Q_P is the square
// root of the largest |(ij|ij)| over the pair's components (the Cauchy-Schwarz bound; the largest
// entry of the positive semidefinite matrix (ab|a'b') lies on its diagonal), computed by the
// library's own FP64 kernels (eri_plan.cu).
//
// Unique quartets: one ordering of each pair of pairs.  The pairs are ranked by decreasing Q
// (ties by increasing P, a stable sort), and the quartet of ranks (r, s) is kept as (bra r, ket
// s) with r <= s.  With a threshold tau the kept kets of bra r are the ranks s >= r with
// Q_r Q_s >= tau; as Q decreases along the ranks they form one contiguous range [r, last(r)],
// found by binary search, so counting, offsets and writing are each one pass over the bras.
// Enumeration order: bra rank ascending, then ket rank ascending; a shard keeps every
// shard_count-th quartet of that sequence starting at shard_index.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include "eri_internal.h"

namespace eri {

namespace {

__device__ __forceinline__ void pair_of(long long P, int &i, int &j) {
    long long a = (long long)((sqrt(8.0 * (double)P + 1.0) - 1.0) * 0.5);
    while ((a + 1) * (a + 2) / 2 <= P) ++a;
    while (a * (a + 1) / 2 > P) --a;
    i = (int)a;
    j = (int)(P - a * (a + 1) / 2);
}

__device__ __forceinline__ long long pair_index(int a, int b) {
    const long long i = a > b ? a : b, j = a > b ? b : a;
    return i * (i + 1) / 2 + j;
}

__global__ void diag_quartets_kernel(long long npairs, int4 *__restrict__ out) {
    for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < npairs;
         P += (long long)gridDim.x * blockDim.x) {
        int i, j;
        pair_of(P, i, j);
        out[P] = make_int4(i, j, i, j);
    }
}

__global__ void iota_kernel(long long n, int *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (int)i;
}

// kets kept for bra rank r (ranks s >= r with Qs[r] Qs[s] >= tau)
__global__ void ket_count_kernel(const double *__restrict__ Qs, long long npairs, double tau,
                                 long long *__restrict__ cnt) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < npairs;
         r += (long long)gridDim.x * blockDim.x) {
        if (!(tau > 0.0)) {
            cnt[r] = npairs - r;
            continue;
        }
        const double qr = Qs[r];
        if (!(qr * Qs[r] >= tau)) {
            cnt[r] = 0;
            continue;
        }
        long long lo = r, hi = npairs - 1;  // invariant: predicate true at lo
        while (lo < hi) {
            const long long mid = lo + (hi - lo + 1) / 2;
            if (qr * Qs[mid] >= tau)
                lo = mid;
            else
                hi = mid - 1;
        }
        cnt[r] = lo - r + 1;
    }
}

// ceil(a / b) for a >= 0, b >= 1, without forming a + b - 1 (b may be close to 2^63)
__host__ __device__ __forceinline__ long long ceil_div_nn(long long a, long long b) {
    return a / b + (a % b != 0 ? 1 : 0);
}

// one warp per bra rank: writes the kept quartets of the shard at their positions.  The bra's
// quartets occupy enumeration positions [o, o + c); the shard keeps t = sidx + m * scount, stored
// at m.  The loop runs over m (no product beyond the enumeration's end is ever formed: m < m1
// implies sidx + m * scount < o + c).
__global__ void unique_write_kernel(const int *__restrict__ pair_rank, const long long *__restrict__ cnt,
                                    const long long *__restrict__ off, long long npairs,
                                    long long sidx, long long scount, int4 *__restrict__ out) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = warp; r < npairs; r += nwarps) {
        const long long c = cnt[r];
        const long long o = off[r];
        const long long end = o + c;
        if (c == 0 || end <= sidx) continue;
        const long long m0 = o > sidx ? ceil_div_nn(o - sidx, scount) : 0;
        const long long m1 = ceil_div_nn(end - sidx, scount);
        int bi, bj;
        pair_of(pair_rank[r], bi, bj);
        for (long long m = m0 + lane; m < m1; m += 32) {
            const long long t = sidx + m * scount;
            const long long s = r + (t - o);
            int ki, kj;
            pair_of(pair_rank[s], ki, kj);
            out[m] = make_int4(bi, bj, ki, kj);
        }
    }
}

__global__ void schwarz_flag_kernel(const int4 *__restrict__ q, long long n, const double *__restrict__ Q,
                                    double tau, char *__restrict__ keep) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 t = q[i];
        keep[i] = Q[pair_index(t.x, t.y)] * Q[pair_index(t.z, t.w)] >= tau ? 1 : 0;
    }
}

// Q_P = sqrt(max |x|) over the n_eri values of each quartet (one warp per quartet)
__global__ void quartet_absmax_sqrt_kernel(const double *__restrict__ x, long long n, int neri,
                                           double *__restrict__ out) {
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= n) return;
    double m = 0.0;
    for (int v = lane; v < neri; v += 32) m = fmax(m, fabs(x[q * neri + v]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) out[q] = sqrt(m);
}

__global__ void scatter_kernel(const double *__restrict__ v, const int *__restrict__ idx, long long n,
                               double *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[idx[i]] = v[i];
}

unsigned grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

cudaError_t screen_diag_quartets(long long npairs, int4 *out, cudaStream_t s) {
    diag_quartets_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(npairs, out);
    return cudaGetLastError();
}

cudaError_t screen_absmax_sqrt(const double *x, long long n, int neri, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    quartet_absmax_sqrt_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(x, n, neri, out);
    return cudaGetLastError();
}

cudaError_t screen_scatter(const double *v, const int *idx, long long n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(v, idx, n, out);
    return cudaGetLastError();
}

cudaError_t screen_unique8(const double *d_Q, long long npairs, double tau, long long sidx,
                           long long scount, int4 **d_out, long long *n_out, long long *total,
                           long long max_out, cudaStream_t s) {
    *d_out = nullptr;
    *n_out = 0;
    *total = 0;
    if (npairs <= 0) return cudaSuccess;
    double *Qs = nullptr;
    int *ids = nullptr, *ranked = nullptr;
    long long *cnt = nullptr, *off = nullptr;
    void *tmp = nullptr;
    size_t tb = 0, tb2 = 0;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMalloc(&Qs, npairs * sizeof(double))) != cudaSuccess) break;
        if ((e = cudaMalloc(&ids, npairs * sizeof(int))) != cudaSuccess) break;
        if ((e = cudaMalloc(&ranked, npairs * sizeof(int))) != cudaSuccess) break;
        if ((e = cudaMalloc(&cnt, npairs * sizeof(long long))) != cudaSuccess) break;
        if ((e = cudaMalloc(&off, npairs * sizeof(long long))) != cudaSuccess) break;
        iota_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(npairs, ids);
        // ranks: decreasing Q, ties in increasing pair index (the radix sort is stable)
        if ((e = cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, d_Q, Qs, ids, ranked, (int)npairs,
                                                           0, 64, s)) != cudaSuccess)
            break;
        if ((e = cub::DeviceScan::ExclusiveSum(nullptr, tb2, cnt, off, (int)npairs, s)) != cudaSuccess) break;
        if ((e = cudaMalloc(&tmp, std::max(tb, tb2))) != cudaSuccess) break;
        if ((e = cub::DeviceRadixSort::SortPairsDescending(tmp, tb, d_Q, Qs, ids, ranked, (int)npairs, 0, 64,
                                                           s)) != cudaSuccess)
            break;
        ket_count_kernel<<<grid_for(npairs, 256), 256, 0, s>>>(Qs, npairs, tau, cnt);
        if ((e = cub::DeviceScan::ExclusiveSum(tmp, tb2, cnt, off, (int)npairs, s)) != cudaSuccess) break;
        long long last[2];
        if ((e = cudaMemcpyAsync(&last[0], off + npairs - 1, sizeof(long long), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(&last[1], cnt + npairs - 1, sizeof(long long), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
            break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        const long long T = last[0] + last[1];
        *total = T;
        const long long kept = T > sidx ? ceil_div_nn(T - sidx, scount) : 0;
        if (kept > max_out) {
            e = cudaErrorNotSupported;  // mapped to ERI_E_UNSUPPORTED by the caller
            break;
        }
        *n_out = kept;
        if (kept == 0) break;
        if ((e = cudaMalloc(d_out, kept * sizeof(int4))) != cudaSuccess) break;
        unique_write_kernel<<<grid_for(npairs * 32, 256), 256, 0, s>>>(ranked, cnt, off, npairs, sidx, scount,
                                                                       *d_out);
        e = cudaGetLastError();
    } while (false);
    cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    cudaFree(Qs);
    cudaFree(ids);
    cudaFree(ranked);
    cudaFree(cnt);
    cudaFree(off);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaFree(*d_out);
        *d_out = nullptr;
        *n_out = 0;
    }
    return e;
}

cudaError_t screen_filter(const int4 *d_in, long long n, const double *d_Q, double tau, int4 **d_out,
                          int **d_idx, long long *n_out, cudaStream_t s) {
    *d_out = nullptr;
    *d_idx = nullptr;
    *n_out = 0;
    if (n <= 0) return cudaSuccess;
    char *keep = nullptr;
    int *iota = nullptr;
    long long *d_n = nullptr;
    void *tmp = nullptr;
    size_t tb = 0, tb2 = 0;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMalloc(&keep, n)) != cudaSuccess) break;
        if ((e = cudaMalloc(&iota, n * sizeof(int))) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_n, sizeof(long long))) != cudaSuccess) break;
        if ((e = cudaMalloc(d_out, n * sizeof(int4))) != cudaSuccess) break;
        if ((e = cudaMalloc(d_idx, n * sizeof(int))) != cudaSuccess) break;
        schwarz_flag_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_in, n, d_Q, tau, keep);
        iota_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, iota);
        if ((e = cub::DeviceSelect::Flagged(nullptr, tb, d_in, keep, *d_out, d_n, (int)n, s)) != cudaSuccess) break;
        if ((e = cub::DeviceSelect::Flagged(nullptr, tb2, iota, keep, *d_idx, d_n, (int)n, s)) != cudaSuccess) break;
        if ((e = cudaMalloc(&tmp, std::max(tb, tb2))) != cudaSuccess) break;
        if ((e = cub::DeviceSelect::Flagged(tmp, tb, d_in, keep, *d_out, d_n, (int)n, s)) != cudaSuccess) break;
        if ((e = cub::DeviceSelect::Flagged(tmp, tb2, iota, keep, *d_idx, d_n, (int)n, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(n_out, d_n, sizeof(long long), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    } while (false);
    cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    cudaFree(keep);
    cudaFree(iota);
    cudaFree(d_n);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaFree(*d_out);
        cudaFree(*d_idx);
        *d_out = nullptr;
        *d_idx = nullptr;
        *n_out = 0;
    }
    return e;
}

}  // namespace eri
