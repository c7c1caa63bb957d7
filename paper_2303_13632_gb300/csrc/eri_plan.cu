// eri_plan.cu -- host side of the C ABI declared in include/eri.h: shell validation and
// normalisation (Sec. II-A), device-side stable sort of quartets by class, the output
// layouts, and the per-class kernel launches.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "eri_internal.h"

namespace eri {

namespace {

LaunchFn g_launch[256 * kNumVariants];
KernelInfo g_info[256 * kNumVariants];
BackwardFn g_backward[256];
BackwardFn g_backward_mixed[256];
std::once_flag g_launch_once;

void register_all() {
    eri_register_backward_0(g_backward, g_backward_mixed);
    eri_register_backward_1(g_backward, g_backward_mixed);
    eri_register_backward_2(g_backward, g_backward_mixed);
    eri_register_backward_3(g_backward, g_backward_mixed);
    eri_register_tu_0(g_launch, g_info); eri_register_tu_1(g_launch, g_info);
    eri_register_tu_2(g_launch, g_info); eri_register_tu_3(g_launch, g_info);
    eri_register_tu_4(g_launch, g_info); eri_register_tu_5(g_launch, g_info);
    eri_register_tu_6(g_launch, g_info); eri_register_tu_7(g_launch, g_info);
    eri_register_tu_8(g_launch, g_info); eri_register_tu_9(g_launch, g_info);
    eri_register_tu_10(g_launch, g_info); eri_register_tu_11(g_launch, g_info);
    eri_register_tu_12(g_launch, g_info); eri_register_tu_13(g_launch, g_info);
    eri_register_tu_14(g_launch, g_info); eri_register_tu_15(g_launch, g_info);
}

int ncart_h(int L) { return (L + 1) * (L + 2) / 2; }

// Axis-aligned normalisation of Sec. II-A:
// N = (2 alpha/pi)^{3/4} (4 alpha)^{L/2} / sqrt((2L-1)!!).
double shell_norm(double alpha, int L) {
    double df = 1.0;
    for (int k = 2 * L - 1; k > 1; k -= 2) df *= k;
    return std::pow(2.0 * alpha / 3.14159265358979323846, 0.75) * std::pow(4.0 * alpha, 0.5 * L) /
           std::sqrt(df);
}

// Canonical representative of a generic class (Sec. II-B, Eq. 3) and the shell permutation:
// canonical slot k takes generic slot perm[k].
struct Canon {
    int cls;
    int perm[4];
    int ostride[4];
};

Canon canonicalise(int cls) {
    int L[4];
    class_ls(cls, L);
    int bra[2] = {0, 1}, ket[2] = {2, 3};
    if (L[0] < L[1]) { bra[0] = 1; bra[1] = 0; }
    if (L[2] < L[3]) { ket[0] = 3; ket[1] = 2; }
    Canon c;
    bool swap = ncart_h(L[bra[0]]) * ncart_h(L[bra[1]]) < ncart_h(L[ket[0]]) * ncart_h(L[ket[1]]);
    int p[4] = {bra[0], bra[1], ket[0], ket[1]};
    if (swap) { p[0] = ket[0]; p[1] = ket[1]; p[2] = bra[0]; p[3] = bra[1]; }
    int gstride[4];
    gstride[3] = 1;
    for (int g = 2; g >= 0; --g) gstride[g] = gstride[g + 1] * ncart_h(L[g + 1]);
    for (int k = 0; k < 4; ++k) {
        c.perm[k] = p[k];
        c.ostride[k] = gstride[p[k]];
    }
    c.cls = class_id_of(L[p[0]], L[p[1]], L[p[2]], L[p[3]]);
    return c;
}

// class key of every quartet: 8 bits when every shell has L <= 3 (ids 0..255), else 10 bits
template <typename K>
__global__ void classify_kernel(const int4 *__restrict__ q, long long n, const int *__restrict__ L,
                                int n_shells, K *__restrict__ keys, int *__restrict__ vals,
                                int *__restrict__ err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 t = q[i];
    bool ok = t.x >= 0 && t.x < n_shells && t.y >= 0 && t.y < n_shells && t.z >= 0 &&
              t.z < n_shells && t.w >= 0 && t.w < n_shells;
    if (!ok) {
        atomicOr(err, 4);
        keys[i] = 0;
    } else {
        keys[i] = (K)class_id_of(L[t.x], L[t.y], L[t.z], L[t.w]);
    }
    vals[i] = (int)i;
}

__global__ void all_quartets_kernel(int n, long long total, int4 *__restrict__ q) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= total) return;
    long long r = i;
    int l = (int)(r % n); r /= n;
    int k = (int)(r % n); r /= n;
    int j = (int)(r % n); r /= n;
    q[i] = make_int4((int)r, j, k, l);
}

__global__ void gather_kernel(const int4 *__restrict__ src, const int *__restrict__ idx,
                              long long n, int4 *__restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

__global__ void check_ids_kernel(const int4 *__restrict__ q, long long n, int n_shells, int *__restrict__ err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 t = q[i];
    if (t.x < 0 || t.x >= n_shells || t.y < 0 || t.y >= n_shells || t.z < 0 || t.z >= n_shells ||
        t.w < 0 || t.w >= n_shells)
        atomicOr(err, 4);
}

__global__ void compose_kernel(int *__restrict__ perm, const int *__restrict__ orig, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = orig[perm[i]];
}

template <typename K>
__global__ void histogram_kernel(const K *__restrict__ keys, long long n,
                                 unsigned long long *__restrict__ counts) {
    __shared__ unsigned int h[kNumClassIds];
    for (int i = threadIdx.x; i < kNumClassIds; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&h[keys[i]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kNumClassIds; i += blockDim.x)
        if (h[i]) atomicAdd(&counts[i], (unsigned long long)h[i]);
}

// Primitive-pair table: record (pa, pb) at (pa * np + pb) * kPairFields holds p = a + b, 1/p,
// P - X = -(b/p)(X - Y) and exp(-ab/p |X - Y|^2) cn_a cn_b for primitives pa of shell X and pb
// of shell Y (Sec. II-A), all in FP64.
__global__ void pair_table_kernel(const double *__restrict__ cx, const double *__restrict__ cy,
                                  const double *__restrict__ cz, const double *__restrict__ exps,
                                  const double *__restrict__ cn, const int *__restrict__ prim_shell,
                                  long long np, double *__restrict__ out) {
    const long long total = np * np;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long pa = i / np, pb = i - pa * np;
        const int x = prim_shell[pa], y = prim_shell[pb];
        const double ea = exps[pa], eb = exps[pb];
        const double p = ea + eb, ip = 1.0 / p;
        const double ab[3] = {cx[x] - cx[y], cy[x] - cy[y], cz[x] - cz[y]};
        const double ab2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
        double *o = out + i * kPairFields;
        o[PR_P] = p;
        o[PR_IP] = ip;
        o[PR_PAX] = -eb * ip * ab[0];
        o[PR_PAY] = -eb * ip * ab[1];
        o[PR_PAZ] = -eb * ip * ab[2];
        o[PR_KCN] = exp(-(ea * eb * ip) * ab2) * cn[pa] * cn[pb];
    }
}

// Largest |b - a| / max|a| over the quartets (a: FP64 values, b: mixed values) of n quartets of
// neri values each; quartets with max|a| <= 1e-30 (below the FP32 range once scaled) are
// skipped.  One warp per quartet; the result (non-negative float) is atomically max-ed in bits.
__global__ void calib_kernel(const double *__restrict__ a, const double *__restrict__ b, long long n,
                             int neri, unsigned int *out) {
    long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int lane = threadIdx.x & 31;
    if (q >= n) return;
    const double *x = a + q * neri, *y = b + q * neri;
    double m = 0.0, d = 0.0;
    for (int i = lane; i < neri; i += 32) {
        m = fmax(m, fabs(x[i]));
        d = fmax(d, fabs(y[i] - x[i]));
    }
    for (int off = 16; off > 0; off >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
        d = fmax(d, __shfl_down_sync(0xffffffffu, d, off));
    }
    if (lane == 0 && m > 1e-30) atomicMax(out, __float_as_uint((float)(d / m)));
}

}  // namespace

}  // namespace eri

using namespace eri;

struct eri_plan_s {
    int device = 0;
    int precision = ERI_FP64;
    int n_shells = 0;
    long long n_prims = 0;
    long long nq = 0;
    long long screen_candidates = 0;  // quartets before Schwarz screening (and sharding)
    long long screen_kept = 0;        // quartets passing the screening, before sharding
    int max_nprim = 1;
    // device arrays
    double *d_cx = nullptr, *d_cy = nullptr, *d_cz = nullptr, *d_exps = nullptr, *d_cn = nullptr;
    int *d_pofs = nullptr, *d_nprim = nullptr;
    int4 *d_quartets = nullptr;  // class-sorted
    int *d_perm = nullptr;       // sorted position -> caller's index
    int *d_err = nullptr;
    int *d_bfoff = nullptr;      // first basis function of every shell
    long long n_bf = 0;          // basis functions (sum of the shells' Cartesian components)
    float *d_D32 = nullptr;      // FP32 copy of the density of eri_digest_jk (lazy)
    void *d_digest = nullptr;    // per-class parameters of eri_digest_jk's launch (lazy)
    void *d_queue = nullptr;     // class table and tile counter of the work-queue launch (lazy)
    void *d_setup = nullptr;      // scratch of the split setup/recurrence path (lazy)
    double *d_pairs = nullptr;    // primitive-pair table (n_prims^2 records), or null
    int *d_prim_shell = nullptr;  // shell of every primitive (with the pair table)
    std::vector<int> h_L, h_nprim;  // per shell, for eri_plan_update_shells
    // batched form: tile counters of the persistent kernels (scratch), streams, graph cache
    unsigned long long *d_counters = nullptr;
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kSide] = {};
    // streamed copies to the host: copy stream and one event per class
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t class_ev[kNumClassIds] = {};
    cudaEvent_t copy_done = nullptr;
    cudaGraphExec_t graph = nullptr;
    int g_bits = -1, g_prec = -1;
    void *g_packed = nullptr;
    float *g_scales = nullptr;
    // per-class precision (-1: the plan's) and the calibrated mixed-path error per class
    int class_prec[kNumClassIds];
    float class_err[kNumClassIds];
    // autotuned launch choice per canonical class and variant (grid 0 = all resident CTAs)
    int tune_phase[256 * kNumVariants] = {0};
    int tune_grid[256 * kNumVariants] = {0};
    // host layout
    long long count[kNumClassIds] = {0};
    long long first[kNumClassIds] = {0};
    long long fp64_off[kNumClassIds] = {0};
    Tables tables;
};

namespace {

void free_plan(eri_plan_s *p) {
    if (!p) return;
    cudaFree(p->d_cx);
    cudaFree(p->d_cy);
    cudaFree(p->d_cz);
    cudaFree(p->d_exps);
    cudaFree(p->d_cn);
    cudaFree(p->d_pofs);
    cudaFree(p->d_nprim);
    cudaFree(p->d_quartets);
    cudaFree(p->d_perm);
    cudaFree(p->d_err);
    cudaFree(p->d_bfoff);
    cudaFree(p->d_D32);
    cudaFree(p->d_digest);
    cudaFree(p->d_queue);
    cudaFree(p->d_setup);
    cudaFree(p->d_pairs);
    cudaFree(p->d_prim_shell);
    cudaFree(p->d_counters);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (int i = 0; i < eri_plan_s::kSide; ++i) {
        if (p->side[i]) cudaStreamDestroy(p->side[i]);
        if (p->join_ev[i]) cudaEventDestroy(p->join_ev[i]);
    }
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    for (int c = 0; c < kNumClassIds; ++c)
        if (p->class_ev[c]) cudaEventDestroy(p->class_ev[c]);
    if (p->copy_done) cudaEventDestroy(p->copy_done);
    delete p;
}

eri_status_t cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return ERI_OK;
    if (e == cudaErrorMemoryAllocation) return ERI_E_NOMEM;
    return ERI_E_CUDA;
}

// Allocation-failure injection for tests of the error paths (no GPU fault involved): with the
// environment variable ERI_INJECT_NOMEM=k (k >= 1) the k-th allocation made by one
// eri_plan_create call (the host plan object first, then its device buffers, in program order,
// including those of the internal plan of diagonal quartets for screening) fails as if memory
// were exhausted.  Read at the start of every eri_plan_create call; unset or 0 = off.
thread_local long long g_inject_nomem = 0;

cudaError_t plan_malloc(void **ptr, size_t bytes) {
    if (g_inject_nomem > 0 && --g_inject_nomem == 0) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}
template <typename T>
cudaError_t plan_malloc(T **ptr, size_t bytes) {
    void *v = nullptr;
    cudaError_t e = plan_malloc(&v, bytes);
    *ptr = static_cast<T *>(v);
    return e;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
    cudaError_t e = plan_malloc(dst, std::max<size_t>(1, src.size()) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Class sort of the plan's quartets on the device: keys (class ids), stable radix sort keeping
// the caller's order within a class, the sorted quartets, the permutation and the class counts.
template <typename K>
cudaError_t class_sort(eri_plan_s *p, const int4 *d_in, long long nq, const int *d_L, int n_shells,
                       const int *d_orig) {
    constexpr int kBits = sizeof(K) == 1 ? 8 : 10;
    cudaError_t e = cudaSuccess;
    K *d_keys = nullptr, *d_keys_sorted = nullptr;
    int *d_vals = nullptr;
    unsigned long long *d_counts = nullptr;
    void *d_tmp = nullptr;
    size_t tmp_bytes = 0;
    int *d_verr = nullptr;
    const unsigned blocks = (unsigned)((nq + 255) / 256);
    do {
        if ((e = plan_malloc(&d_keys, nq * sizeof(K))) != cudaSuccess) break;
        if ((e = plan_malloc(&d_keys_sorted, nq * sizeof(K))) != cudaSuccess) break;
        if ((e = plan_malloc(&d_vals, nq * sizeof(int))) != cudaSuccess) break;
        if ((e = plan_malloc(&p->d_perm, nq * sizeof(int))) != cudaSuccess) break;
        if ((e = plan_malloc(&d_verr, sizeof(int))) != cudaSuccess) break;
        if ((e = cudaMemset(d_verr, 0, sizeof(int))) != cudaSuccess) break;
        classify_kernel<K><<<blocks, 256>>>(d_in, nq, d_L, n_shells, d_keys, d_vals, d_verr);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // stable radix sort on the class key keeps the caller's order within a class
        e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, d_keys, d_keys_sorted, d_vals,
                                            p->d_perm, (int)nq, 0, kBits);
        if (e != cudaSuccess) break;
        if ((e = plan_malloc(&d_tmp, std::max<size_t>(tmp_bytes, 1))) != cudaSuccess) break;
        e = cub::DeviceRadixSort::SortPairs(d_tmp, tmp_bytes, d_keys, d_keys_sorted, d_vals,
                                            p->d_perm, (int)nq, 0, kBits);
        if (e != cudaSuccess) break;
        if ((e = plan_malloc(&p->d_quartets, nq * sizeof(int4))) != cudaSuccess) break;
        gather_kernel<<<blocks, 256>>>(d_in, p->d_perm, nq, p->d_quartets);
        if ((e = plan_malloc(&d_counts, kNumClassIds * sizeof(unsigned long long))) != cudaSuccess) break;
        if ((e = cudaMemset(d_counts, 0, kNumClassIds * sizeof(unsigned long long))) != cudaSuccess) break;
        histogram_kernel<K><<<std::min<unsigned>(blocks, 4096u), 256>>>(d_keys_sorted, nq, d_counts);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        unsigned long long counts[kNumClassIds];
        if ((e = cudaMemcpy(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
        int verr = 0;
        if ((e = cudaMemcpy(&verr, d_verr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
            break;
        if (verr) e = cudaErrorInvalidValue;  // mapped to ERI_E_INVALID below
        for (int c = 0; c < kNumClassIds; ++c) p->count[c] = (long long)counts[c];
        if (d_orig) {  // sorted position -> index in the caller's list
            compose_kernel<<<blocks, 256>>>(p->d_perm, d_orig, nq);
            e = cudaGetLastError();
        }
    } while (false);
    cudaError_t sync_e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = sync_e;
    cudaFree(d_keys);
    cudaFree(d_keys_sorted);
    cudaFree(d_vals);
    cudaFree(d_counts);
    cudaFree(d_tmp);
    cudaFree(d_verr);
    return e;
}

size_t packed_segment_bytes(long long nq, int neri, int bits) {
    unsigned long long b = ((unsigned long long)nq * neri * bits + 7) / 8;
    return (size_t)((b + 255) / 256 * 256);
}

// Bytes of one class in the paper's chunk layout: n_CS = ceil(n_eri / floor(512/bits)) 64-byte
// chunks per quartet (Sec. III-C).
size_t paper512_segment_bytes(long long nq, int neri, int bits) {
    const long long F = 512 / bits;
    return (size_t)nq * (size_t)((neri + F - 1) / F) * 64;
}

int class_neri(int cls) {
    int L[4];
    class_ls(cls, L);
    return ncart_h(L[0]) * ncart_h(L[1]) * ncart_h(L[2]) * ncart_h(L[3]);
}

// bytes of the plan's scratch (split setup records, or the FP64 values of the compressed output
// of classes with a g shell)
constexpr size_t kScratchBytes = (size_t)kSetupChunk * kSetupFieldsMax * sizeof(double);

cudaError_t ensure_scratch(eri_plan_s *p) {
    return p->d_setup ? cudaSuccess : cudaMalloc(&p->d_setup, kScratchBytes);
}

int class_precision(const eri_plan_s *p, int cls) {
    return p->class_prec[cls] >= 0 ? p->class_prec[cls] : p->precision;
}

int class_variant(const eri_plan_s *p, int cls) {
    return class_precision(p, cls) == ERI_FP64 ? 0 : (p->max_nprim > 1 ? 2 : 1);
}

ClassArgs class_args(eri_plan_s *p, int cls, double *d_out, int bits, void *d_packed, float *d_scales,
                     size_t packed_off) {
    Canon c = canonicalise(cls);
    ClassArgs a{};
    for (int k = 0; k < 4; ++k) {
        a.perm[k] = c.perm[k];
        a.ostride[k] = c.ostride[k];
    }
    a.quartets = p->d_quartets + p->first[cls];
    a.nq = p->count[cls];
    a.err = p->d_err;
    a.pairs = p->d_pairs;
    a.np = p->n_prims;
    int neri = class_neri(cls);
    if (d_out) {
        a.out_fp64 = d_out + p->fp64_off[cls];
    } else {
        a.packed = reinterpret_cast<uint32_t *>(static_cast<char *>(d_packed) + packed_off);
        a.seg_words = (long long)(packed_segment_bytes(p->count[cls], neri, bits) / 4);
        a.scales = d_scales + p->first[cls];
        a.bits = bits;
    }
    return a;
}

// Launches the kernels of generic class cls with prepared arguments `a` (its quartets, count
// and output) in precision variant `variant`; primitive plans run the split setup/recurrence
// path in chunks of kSetupChunk quartets where the class has no thread-per-quartet form.
eri_status_t launch_class_args(eri_plan_s *p, int cls, const ClassArgs &a, int variant,
                               cudaStream_t stream) {
    if (a.nq == 0) return ERI_OK;
    Canon c = canonicalise(cls);
    ShellsDev sh{p->d_cx, p->d_cy, p->d_cz, p->d_pofs, p->d_nprim, p->d_exps, p->d_cn};
    const int neri = class_neri(cls);
    const int bits = a.bits;
    if (class_has_g(c.cls)) {
        int L[4];
        class_ls(c.cls, L);
        if (!a.out_fp64) {
            cudaError_t e = ensure_scratch(p);
            if (e != cudaSuccess) return cuda_status(e);
        }
        return cuda_status(launch_generic(sh, p->tables, a, L, variant != 0, static_cast<double *>(p->d_setup),
                                          kScratchBytes, stream));
    }
    LaunchFn fn = g_launch[c.cls * kNumVariants + variant];
    if (!fn) return ERI_E_UNSUPPORTED;
    LaunchOpts o;
    o.device = p->device;
    const bool split = p->max_nprim == 1 && g_info[c.cls * kNumVariants + variant].setup;
    if (!split) return cuda_status(fn(sh, p->tables, a, stream, o));
    {
        cudaError_t e = ensure_scratch(p);
        if (e != cudaSuccess) return cuda_status(e);
    }
    o.scratch = p->d_setup;
    // chunks of kSetupChunk quartets (multiples of 32: every chunk starts on a packed word)
    for (long long c0 = 0; c0 < a.nq; c0 += kSetupChunk) {
        ClassArgs ac = a;
        ac.quartets = a.quartets + c0;
        ac.nq = std::min<long long>(kSetupChunk, a.nq - c0);
        if (a.out_fp64) {
            ac.out_fp64 = a.out_fp64 + c0 * neri;
        } else {
            long long w = c0 * neri * bits / 32;
            ac.packed = a.packed + w;
            ac.scales = a.scales + c0;
            ac.seg_words = (c0 + ac.nq == a.nq) ? a.seg_words - w : ac.nq * neri * bits / 32;
        }
        cudaError_t e = fn(sh, p->tables, ac, stream, o);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return ERI_OK;
}

// Schwarz factors Q[P] = sqrt(max |(ij|ij)|) of every unordered shell pair P = i (i + 1) / 2 + j
// (i >= j): FP64 ERIs of the diagonal quartets by the library's own kernels (a plan of those
// quartets), computed class by class in chunks of a bounded buffer and reduced on the device.
// *d_Q (npairs doubles) is allocated here.
eri_status_t schwarz_factors(const eri_shell_t *shells, int n_shells, int device, int flags, double **d_Q) {
    *d_Q = nullptr;
    const long long npairs = (long long)n_shells * (n_shells + 1) / 2;
    if (npairs == 0) return ERI_OK;
    constexpr long long kChunkDoubles = 1LL << 25;  // 256 MiB of FP64 output per launch
    int4 *d_diag = nullptr;
    double *Qs = nullptr, *buf = nullptr;
    eri_plan_t sp = nullptr;
    cudaError_t e = plan_malloc(&d_diag, npairs * sizeof(int4));
    if (e == cudaSuccess) e = screen_diag_quartets(npairs, d_diag, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d_diag);
        return cuda_status(e);
    }
    eri_plan_opts_t so{ERI_FP64, ERI_EXPLICIT, device, ERI_QUARTETS_ON_DEVICE | flags, 0.0, 0, 0};
    eri_status_t st = eri_plan_create(shells, n_shells, reinterpret_cast<const int32_t *>(d_diag), npairs, &so, &sp);
    cudaFree(d_diag);
    if (st != ERI_OK) return st;
    long long maxv = 1;
    for (int c = 0; c < kNumClassIds; ++c)
        if (sp->count[c] > 0) maxv = std::max(maxv, std::min(sp->count[c], std::max(1LL, kChunkDoubles / class_neri(c))) * class_neri(c));
    e = plan_malloc(&Qs, npairs * sizeof(double));
    if (e == cudaSuccess) e = plan_malloc(&buf, maxv * sizeof(double));
    if (e == cudaSuccess) e = plan_malloc(d_Q, npairs * sizeof(double));
    for (int c = 0; e == cudaSuccess && st == ERI_OK && c < kNumClassIds; ++c) {
        if (sp->count[c] == 0) continue;
        const int neri = class_neri(c);
        const long long chunk = std::max(1LL, kChunkDoubles / neri);
        for (long long c0 = 0; c0 < sp->count[c] && st == ERI_OK; c0 += chunk) {
            ClassArgs a = class_args(sp, c, buf, 0, nullptr, nullptr, 0);
            a.quartets += c0;
            a.nq = std::min(chunk, sp->count[c] - c0);
            a.out_fp64 = buf;
            st = launch_class_args(sp, c, a, 0, nullptr);
            if (st == ERI_OK) e = screen_absmax_sqrt(buf, a.nq, neri, Qs + sp->first[c] + c0, nullptr);
            if (e != cudaSuccess) st = cuda_status(e);
        }
    }
    if (st == ERI_OK && e == cudaSuccess) e = screen_scatter(Qs, sp->d_perm, npairs, *d_Q, nullptr);
    cudaError_t se = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = se;
    if (st == ERI_OK && e != cudaSuccess) st = cuda_status(e);
    cudaFree(Qs);
    cudaFree(buf);
    eri_plan_destroy(sp);
    if (st != ERI_OK) {
        cudaFree(*d_Q);
        *d_Q = nullptr;
    }
    return st;
}

eri_status_t launch_one(eri_plan_s *p, int cls, double *d_out, int bits, void *d_packed,
                        float *d_scales, size_t packed_off, cudaStream_t stream) {
    if (p->count[cls] == 0) return ERI_OK;
    ClassArgs a = class_args(p, cls, d_out, bits, d_packed, d_scales, packed_off);
    return launch_class_args(p, cls, a, class_variant(p, cls), stream);
}

eri_status_t ensure_batched_resources(eri_plan_s *p) {
    cudaError_t e = cudaSuccess;
    if (!p->d_counters) e = cudaMalloc(&p->d_counters, 256 * sizeof(unsigned long long));
    bool has_g = false;
    for (int c = 256; c < kNumClassIds; ++c) has_g |= p->count[c] > 0;
    if (e == cudaSuccess && has_g) e = ensure_scratch(p);  // before any stream capture
    for (int i = 0; e == cudaSuccess && i < eri_plan_s::kSide; ++i) {
        if (!p->side[i]) e = cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess && !p->join_ev[i])
            e = cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !p->fork_ev) e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming);
    return cuda_status(e);
}

// Persistent launches of every non-empty class on the plan's side streams (forked from and
// joined back into `stream`); the classes go to the side streams by decreasing quartet count.
eri_status_t enqueue_batched(eri_plan_s *p, int bits, void *d_packed, float *d_scales,
                             cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(p->d_counters, 0, 256 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->fork_ev, stream);
    for (int i = 0; e == cudaSuccess && i < eri_plan_s::kSide; ++i)
        e = cudaStreamWaitEvent(p->side[i], p->fork_ev, 0);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<int> cls;
    std::vector<size_t> off(kNumClassIds, 0);
    size_t o = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        off[c] = o;
        o += packed_segment_bytes(p->count[c], class_neri(c), bits);
        if (p->count[c] > 0) cls.push_back(c);
    }
    std::sort(cls.begin(), cls.end(), [&](int x, int y) {
        return p->count[x] * class_neri(x) > p->count[y] * class_neri(y);
    });
    ShellsDev sh{p->d_cx, p->d_cy, p->d_cz, p->d_pofs, p->d_nprim, p->d_exps, p->d_cn};
    for (size_t i = 0; i < cls.size(); ++i) {
        int c = cls[i];
        int cc = canonicalise(c).cls;
        const int variant = class_variant(p, c);
        if (class_has_g(cc)) {
            // plain launches of the run-time-L kernels; all on the first side stream, since
            // they share the plan's scratch
            ClassArgs a = class_args(p, c, nullptr, bits, d_packed, d_scales, off[c]);
            eri_status_t st = launch_class_args(p, c, a, variant, p->side[0]);
            if (st != ERI_OK) return st;
            continue;
        }
        LaunchFn fn = g_launch[cc * kNumVariants + variant];
        if (!fn) return ERI_E_UNSUPPORTED;
        ClassArgs a = class_args(p, c, nullptr, bits, d_packed, d_scales, off[c]);
        LaunchOpts lo;
        lo.device = p->device;
        lo.counter = p->d_counters + c;
        lo.force_phase = p->tune_phase[cc * kNumVariants + variant];
        lo.grid = p->tune_grid[cc * kNumVariants + variant];
        e = fn(sh, p->tables, a, p->side[i % eri_plan_s::kSide], lo);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int i = 0; e == cudaSuccess && i < eri_plan_s::kSide; ++i) {
        e = cudaEventRecord(p->join_ev[i], p->side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, p->join_ev[i], 0);
    }
    return cuda_status(e);
}

}  // namespace

extern "C" {

const char *eri_status_string(eri_status_t s) {
    switch (s) {
        case ERI_OK: return "ERI_OK";
        case ERI_E_INVALID: return "ERI_E_INVALID";
        case ERI_E_UNSUPPORTED: return "ERI_E_UNSUPPORTED";
        case ERI_E_NOMEM: return "ERI_E_NOMEM";
        case ERI_E_CUDA: return "ERI_E_CUDA";
        case ERI_E_NUMERIC: return "ERI_E_NUMERIC";
    }
    return "ERI_E_UNKNOWN";
}

int32_t eri_class_id(int32_t La, int32_t Lb, int32_t Lc, int32_t Ld) {
    if (La < 0 || La > kLmax || Lb < 0 || Lb > kLmax || Lc < 0 || Lc > kLmax || Ld < 0 || Ld > kLmax)
        return -1;
    return class_id_of(La, Lb, Lc, Ld);
}

eri_status_t eri_class_shape(int32_t cls, int32_t *n_eri, int32_t *n_rys) {
    if (!class_id_valid(cls)) return ERI_E_INVALID;
    int L[4];
    class_ls(cls, L);
    if (n_eri) *n_eri = ncart_h(L[0]) * ncart_h(L[1]) * ncart_h(L[2]) * ncart_h(L[3]);
    if (n_rys) *n_rys = (L[0] + L[1] + L[2] + L[3]) / 2 + 1;
    return ERI_OK;
}

eri_status_t eri_plan_create(const eri_shell_t *shells, int32_t n_shells, const int32_t *quartets,
                             int64_t n_quartets, const eri_plan_opts_t *opts, eri_plan_t *out) {
    if (!out || (!shells && n_shells > 0) || n_shells < 0) return ERI_E_INVALID;
    eri_plan_opts_t o{ERI_FP64, ERI_EXPLICIT, 0, 0, 0.0, 0, 0};
    if (opts) o = *opts;
    if (o.precision != ERI_FP64 && o.precision != ERI_MIXED) return ERI_E_INVALID;
    if (o.quartet_mode != ERI_EXPLICIT && o.quartet_mode != ERI_ALL && o.quartet_mode != ERI_UNIQUE8)
        return ERI_E_INVALID;
    if (o.flags & ~(ERI_QUARTETS_ON_DEVICE | ERI_NO_PAIR_TABLE)) return ERI_E_INVALID;
    if (!(o.schwarz_threshold >= 0.0) || !std::isfinite(o.schwarz_threshold)) return ERI_E_INVALID;
    const long long scount = o.shard_count > 1 ? o.shard_count : 1;
    if (o.shard_count < 0 || (scount > 1 && o.quartet_mode != ERI_UNIQUE8) || o.shard_index < 0 ||
        o.shard_index >= scount)
        return ERI_E_INVALID;
    const bool screen = o.schwarz_threshold > 0.0;
    const long long npairs = (long long)n_shells * (n_shells + 1) / 2;
    if ((screen || o.quartet_mode == ERI_UNIQUE8) && npairs >= 2147483647LL) return ERI_E_UNSUPPORTED;
    long long nq = 0;
    if (o.quartet_mode == ERI_UNIQUE8) {
        nq = 0;  // known after the enumeration
    } else if (o.quartet_mode == ERI_ALL) {
        double t = (double)n_shells * n_shells * n_shells * n_shells;
        if (t >= 2147483647.0) return ERI_E_UNSUPPORTED;
        nq = (long long)n_shells * n_shells * n_shells * n_shells;
    } else {
        if (n_quartets < 0 || (n_quartets > 0 && !quartets)) return ERI_E_INVALID;
        if (n_quartets >= 2147483647LL) return ERI_E_UNSUPPORTED;
        nq = n_quartets;
    }
    // host validation and normalisation of the shells
    std::vector<double> cx(n_shells), cy(n_shells), cz(n_shells), ex, cn;
    std::vector<int> pofs(n_shells), np(n_shells), Ls(n_shells), bfoff(n_shells);
    int max_nprim = 1;
    long long n_bf = 0;
    for (int s = 0; s < n_shells; ++s) {
        const eri_shell_t &sh = shells[s];
        if (sh.L < 0 || sh.L > kLmax) return sh.L > kLmax ? ERI_E_UNSUPPORTED : ERI_E_INVALID;
        if (sh.nprim < 1 || !sh.exps || !sh.coefs) return ERI_E_INVALID;
        for (int x = 0; x < 3; ++x)
            if (!std::isfinite(sh.center[x])) return ERI_E_INVALID;
        cx[s] = sh.center[0];
        cy[s] = sh.center[1];
        cz[s] = sh.center[2];
        pofs[s] = (int)ex.size();
        np[s] = sh.nprim;
        Ls[s] = sh.L;
        bfoff[s] = (int)n_bf;
        n_bf += ncart_h(sh.L);
        max_nprim = std::max(max_nprim, sh.nprim);
        for (int k = 0; k < sh.nprim; ++k) {
            double a = sh.exps[k], c = sh.coefs[k];
            if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(c)) return ERI_E_INVALID;
            ex.push_back(a);
            cn.push_back(c * shell_norm(a, sh.L));
        }
    }
    if (ex.size() >= 2147483647ull || n_bf >= 2147483647LL) return ERI_E_UNSUPPORTED;
    std::call_once(g_launch_once, register_all);
    {
        const char *inj = std::getenv("ERI_INJECT_NOMEM");
        g_inject_nomem = inj ? std::atoll(inj) : 0;
    }
    if (g_inject_nomem > 0 && --g_inject_nomem == 0) return ERI_E_NOMEM;  // the host plan object
    eri_plan_s *p = new (std::nothrow) eri_plan_s();
    if (!p) return ERI_E_NOMEM;

    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
        delete p;
        return ERI_E_INVALID;
    }
    // Schwarz factors of every shell pair (Sec. II-B bound), for screening and for the ranks of
    // the unique-quartet enumeration (all zero without screening: ranks in pair order)
    double *d_Q = nullptr;
    if (screen) {
        const long long inject = g_inject_nomem;  // the internal plan restarts the count
        eri_status_t st = schwarz_factors(shells, n_shells, o.device, o.flags & ERI_NO_PAIR_TABLE, &d_Q);
        g_inject_nomem = inject;
        if (st != ERI_OK) {
            delete p;
            return st;
        }
    } else if (o.quartet_mode == ERI_UNIQUE8 && npairs > 0) {
        if ((e = plan_malloc(&d_Q, npairs * sizeof(double))) == cudaSuccess)
            e = cudaMemset(d_Q, 0, npairs * sizeof(double));
        if (e != cudaSuccess) {
            cudaFree(d_Q);
            delete p;
            return cuda_status(e);
        }
    }
    p->device = o.device;
    p->precision = o.precision;
    p->n_shells = n_shells;
    p->n_prims = (long long)ex.size();
    p->nq = nq;
    p->max_nprim = max_nprim;
    p->n_bf = n_bf;
    p->h_L = Ls;
    p->h_nprim = np;
    for (int c = 0; c < kNumClassIds; ++c) {
        p->class_prec[c] = -1;
        p->class_err[c] = -1.0f;
    }
    if ((e = tables_for_current_device(&p->tables)) != cudaSuccess) { free_plan(p); return cuda_status(e); }
    int *d_L = nullptr;
    e = upload(&p->d_cx, cx);
    if (e == cudaSuccess) e = upload(&p->d_cy, cy);
    if (e == cudaSuccess) e = upload(&p->d_cz, cz);
    if (e == cudaSuccess) e = upload(&p->d_exps, ex);
    if (e == cudaSuccess) e = upload(&p->d_cn, cn);
    if (e == cudaSuccess) e = upload(&p->d_pofs, pofs);
    if (e == cudaSuccess) e = upload(&p->d_nprim, np);
    if (e == cudaSuccess) e = upload(&d_L, Ls);
    if (e == cudaSuccess) e = upload(&p->d_bfoff, bfoff);
    if (e == cudaSuccess) e = plan_malloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) { cudaFree(d_L); cudaFree(d_Q); free_plan(p); return cuda_status(e); }

    // the quartet list on the device: d_in (owned unless it is the caller's device list) and,
    // for a screened caller's list, the caller's index of every kept quartet (d_orig)
    int4 *d_in = nullptr;
    int *d_orig = nullptr;
    bool own_in = true;
    if (o.quartet_mode == ERI_UNIQUE8) {
        long long total = 0;
        e = screen_unique8(d_Q, npairs, o.schwarz_threshold, o.shard_index, scount, &d_in, &nq, &total,
                           2147483646LL, nullptr);
        p->screen_candidates = npairs * (npairs + 1) / 2;
        p->screen_kept = total;
    } else if (nq > 0) {
        const unsigned blocks = (unsigned)((nq + 255) / 256);
        if (o.quartet_mode == ERI_ALL) {
            if ((e = plan_malloc(&d_in, nq * sizeof(int4))) == cudaSuccess) {
                all_quartets_kernel<<<blocks, 256>>>(n_shells, nq, d_in);
                e = cudaGetLastError();
            }
        } else if (o.flags & ERI_QUARTETS_ON_DEVICE) {
            d_in = reinterpret_cast<int4 *>(const_cast<int32_t *>(quartets));
            own_in = false;
        } else {
            if ((e = plan_malloc(&d_in, nq * sizeof(int4))) == cudaSuccess)
                e = cudaMemcpy(d_in, quartets, nq * sizeof(int4), cudaMemcpyHostToDevice);
        }
        p->screen_candidates = nq;
        p->screen_kept = nq;
        if (e == cudaSuccess && screen) {
            // ids are validated before they index the pair factors
            int *d_verr = nullptr;
            if ((e = plan_malloc(&d_verr, sizeof(int))) == cudaSuccess &&
                (e = cudaMemset(d_verr, 0, sizeof(int))) == cudaSuccess) {
                check_ids_kernel<<<blocks, 256>>>(d_in, nq, n_shells, d_verr);
                int verr = 0;
                if ((e = cudaMemcpy(&verr, d_verr, sizeof(int), cudaMemcpyDeviceToHost)) == cudaSuccess && verr)
                    e = cudaErrorInvalidValue;
            }
            cudaFree(d_verr);
            int4 *d_f = nullptr;
            long long nf = 0;
            if (e == cudaSuccess) e = screen_filter(d_in, nq, d_Q, o.schwarz_threshold, &d_f, &d_orig, &nf, nullptr);
            if (e == cudaSuccess) {
                if (own_in) cudaFree(d_in);
                d_in = d_f;
                own_in = true;
                nq = nf;
                p->screen_kept = nf;
            }
        }
    }
    cudaFree(d_Q);
    p->nq = nq;
    if (e != cudaSuccess) {
        if (own_in) cudaFree(d_in);
        cudaFree(d_orig);
        cudaFree(d_L);
        free_plan(p);
        return e == cudaErrorInvalidValue ? ERI_E_INVALID
                                          : (e == cudaErrorNotSupported ? ERI_E_UNSUPPORTED : cuda_status(e));
    }

    if (nq > 0) {
        const bool g = std::find_if(Ls.begin(), Ls.end(), [](int l) { return l > 3; }) != Ls.end();
        e = g ? class_sort<uint16_t>(p, d_in, nq, d_L, n_shells, d_orig)
              : class_sort<uint8_t>(p, d_in, nq, d_L, n_shells, d_orig);
        cudaError_t sync_e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = sync_e;
        if (own_in) cudaFree(d_in);
        if (e != cudaSuccess) {
            cudaFree(d_orig);
            cudaFree(d_L);
            free_plan(p);
            return e == cudaErrorInvalidValue ? ERI_E_INVALID : cuda_status(e);
        }
    } else if (own_in) {
        cudaFree(d_in);
    }
    cudaFree(d_orig);
    cudaFree(d_L);
    // primitive-pair table, when it fits: n_prims^2 records of kPairFields doubles
    if (!(o.flags & ERI_NO_PAIR_TABLE) && p->nq > 0) {
        const double bytes = (double)p->n_prims * (double)p->n_prims * kPairFields * sizeof(double);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
        if (bytes <= (double)kPairTableMaxBytes && bytes <= 0.25 * (double)free_b) {
            std::vector<int> prim_shell(ex.size());
            for (int s2 = 0; s2 < n_shells; ++s2)
                for (int k = 0; k < shells[s2].nprim; ++k) prim_shell[pofs[s2] + k] = s2;
            int *d_ps = nullptr;
            cudaError_t pe = upload(&d_ps, prim_shell);
            if (pe == cudaSuccess) pe = plan_malloc(&p->d_pairs, (size_t)bytes);
            if (pe == cudaSuccess) {
                pair_table_kernel<<<4 * 1024, 256>>>(p->d_cx, p->d_cy, p->d_cz, p->d_exps, p->d_cn,
                                                      d_ps, p->n_prims, p->d_pairs);
                pe = cudaGetLastError();
                if (pe == cudaSuccess) pe = cudaDeviceSynchronize();
            }
            p->d_prim_shell = d_ps;  // kept: eri_plan_update_shells rebuilds the table
            if (pe != cudaSuccess) {
                free_plan(p);
                return cuda_status(pe);
            }
        }
    }
    long long f = 0, off = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        p->first[c] = f;
        p->fp64_off[c] = off;
        const int neri = class_neri(c);
        f += p->count[c];
        off += p->count[c] * neri;
    }
    *out = p;
    return ERI_OK;
}

void eri_plan_destroy(eri_plan_t plan) {
    if (!plan) return;
    cudaSetDevice(plan->device);
    free_plan(plan);
}

eri_status_t eri_plan_update_shells(eri_plan_t plan, const eri_shell_t *shells, int32_t n_shells,
                                    void *stream) {
    if (!plan || !shells || n_shells != plan->n_shells) return ERI_E_INVALID;
    std::vector<double> cx(n_shells), cy(n_shells), cz(n_shells), ex, cn;
    ex.reserve((size_t)plan->n_prims);
    cn.reserve((size_t)plan->n_prims);
    for (int s = 0; s < n_shells; ++s) {
        const eri_shell_t &sh = shells[s];
        if (sh.L != plan->h_L[s] || sh.nprim != plan->h_nprim[s] || !sh.exps || !sh.coefs)
            return ERI_E_INVALID;
        for (int x = 0; x < 3; ++x)
            if (!std::isfinite(sh.center[x])) return ERI_E_INVALID;
        cx[s] = sh.center[0];
        cy[s] = sh.center[1];
        cz[s] = sh.center[2];
        for (int k = 0; k < sh.nprim; ++k) {
            const double a = sh.exps[k], c = sh.coefs[k];
            if (!(a > 0.0) || !std::isfinite(a) || !std::isfinite(c)) return ERI_E_INVALID;
            ex.push_back(a);
            cn.push_back(c * shell_norm(a, sh.L));
        }
    }
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_status(e);
    if (n_shells == 0) return ERI_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // stream-ordered after the plan's earlier work on `stream`; the host vectors live until the
    // stream has consumed them (synchronised below)
    const size_t sb = n_shells * sizeof(double), pb = ex.size() * sizeof(double);
    e = cudaMemcpyAsync(plan->d_cx, cx.data(), sb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_cy, cy.data(), sb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_cz, cz.data(), sb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_exps, ex.data(), pb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(plan->d_cn, cn.data(), pb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && plan->d_pairs) {
        pair_table_kernel<<<4 * 1024, 256, 0, st>>>(plan->d_cx, plan->d_cy, plan->d_cz, plan->d_exps,
                                                      plan->d_cn, plan->d_prim_shell, plan->n_prims,
                                                      plan->d_pairs);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = se;
    return cuda_status(e);
}

eri_status_t eri_plan_set_precision(eri_plan_t plan, int32_t precision) {
    if (!plan || (precision != ERI_FP64 && precision != ERI_MIXED)) return ERI_E_INVALID;
    plan->precision = precision;
    return ERI_OK;
}

eri_status_t eri_plan_set_class_precision(eri_plan_t plan, int32_t cls, int32_t precision) {
    if (!plan || !class_id_valid(cls)) return ERI_E_INVALID;
    if (precision != ERI_FP64 && precision != ERI_MIXED && precision != -1) return ERI_E_INVALID;
    plan->class_prec[cls] = precision;
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    return ERI_OK;
}

eri_status_t eri_plan_class_precision(eri_plan_t plan, int32_t cls, int32_t *precision,
                                      float *mixed_err) {
    if (!plan || !class_id_valid(cls)) return ERI_E_INVALID;
    if (precision) *precision = class_precision(plan, cls);
    if (mixed_err) *mixed_err = plan->class_err[cls];
    return ERI_OK;
}

eri_status_t eri_plan_num_quartets(eri_plan_t plan, int64_t *n) {
    if (!plan || !n) return ERI_E_INVALID;
    *n = plan->nq;
    return ERI_OK;
}

eri_status_t eri_plan_class_info(eri_plan_t plan, int32_t cls, int64_t *n_quartets,
                                 int32_t *n_eri_per_quartet, int64_t *first_quartet,
                                 int64_t *fp64_offset) {
    if (!plan || !class_id_valid(cls)) return ERI_E_INVALID;
    if (n_quartets) *n_quartets = plan->count[cls];
    if (n_eri_per_quartet) eri_class_shape(cls, n_eri_per_quartet, nullptr);
    if (first_quartet) *first_quartet = plan->first[cls];
    if (fp64_offset) *fp64_offset = plan->fp64_off[cls];
    return ERI_OK;
}

eri_status_t eri_plan_quartet_order(eri_plan_t plan, int64_t *perm_out) {
    if (!plan || (!perm_out && plan->nq > 0)) return ERI_E_INVALID;
    if (plan->nq == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    std::vector<int> tmp(plan->nq);
    cudaError_t e = cudaMemcpy(tmp.data(), plan->d_perm, plan->nq * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    for (long long i = 0; i < plan->nq; ++i) perm_out[i] = tmp[i];
    return ERI_OK;
}

eri_status_t eri_packed_class_offset(eri_plan_t plan, int32_t bits, int32_t cls,
                                     size_t *byte_offset, size_t *bytes) {
    if (!plan || !class_id_valid(cls) || bits < 2 || bits > 24) return ERI_E_INVALID;
    size_t off = 0;
    for (int c = 0; c < cls; ++c) off += packed_segment_bytes(plan->count[c], class_neri(c), bits);
    if (byte_offset) *byte_offset = off;
    if (bytes) *bytes = packed_segment_bytes(plan->count[cls], class_neri(cls), bits);
    return ERI_OK;
}

eri_status_t eri_output_bytes(eri_plan_t plan, int32_t bits, size_t *packed_bytes,
                              size_t *scales_bytes) {
    if (!plan || (bits != 0 && (bits < 2 || bits > 24))) return ERI_E_INVALID;
    size_t total = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        const int neri = class_neri(c);
        total += bits == 0 ? (size_t)plan->count[c] * neri * sizeof(double)
                           : packed_segment_bytes(plan->count[c], neri, bits);
    }
    if (packed_bytes) *packed_bytes = total;
    if (scales_bytes) *scales_bytes = bits == 0 ? 0 : (size_t)plan->nq * sizeof(float);
    return ERI_OK;
}

eri_status_t eri_paper512_class_offset(eri_plan_t plan, int32_t bits, int32_t cls,
                                       size_t *byte_offset, size_t *bytes) {
    if (!plan || (cls != kNumClassIds && !class_id_valid(cls)) || bits < 2 || bits > 24) return ERI_E_INVALID;
    size_t off = 0;
    for (int c = 0; c < cls; ++c) off += paper512_segment_bytes(plan->count[c], class_neri(c), bits);
    if (byte_offset) *byte_offset = off;
    if (bytes) *bytes = cls == kNumClassIds ? 0 : paper512_segment_bytes(plan->count[cls], class_neri(cls), bits);
    return ERI_OK;
}

eri_status_t eri_pack_paper512(eri_plan_t plan, int32_t bits, const void *d_packed, void *d_chunks,
                               void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_chunks)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_chunks) % 4)
        return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    size_t in = 0, out = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        const int neri = class_neri(c);
        if (plan->count[c] > 0) {
            eri_status_t st = eri_pack_paper512_stream(static_cast<const char *>(d_packed) + in,
                                                       plan->count[c], neri, bits,
                                                       static_cast<char *>(d_chunks) + out, stream);
            if (st != ERI_OK) return st;
        }
        in += packed_segment_bytes(plan->count[c], neri, bits);
        out += paper512_segment_bytes(plan->count[c], neri, bits);
    }
    return ERI_OK;
}

eri_status_t eri_compute_class(eri_plan_t plan, int32_t cls, double *d_out, void *stream) {
    if (!plan || !class_id_valid(cls) || (!d_out && plan->nq > 0)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_out) % 8) return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    return launch_one(plan, cls, d_out, 0, nullptr, nullptr, 0, (cudaStream_t)stream);
}

eri_status_t eri_compute(eri_plan_t plan, double *d_out, void *stream) {
    if (!plan || (!d_out && plan->nq > 0)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_out) % 8) return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    for (int c = 0; c < kNumClassIds; ++c) {
        eri_status_t s = launch_one(plan, c, d_out, 0, nullptr, nullptr, 0, (cudaStream_t)stream);
        if (s != ERI_OK) return s;
    }
    return ERI_OK;
}

eri_status_t eri_compute_compressed_class(eri_plan_t plan, int32_t cls, int32_t bits,
                                          void *d_packed, float *d_scales, void *stream) {
    if (!plan || !class_id_valid(cls) || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4)
        return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    size_t off = 0;
    eri_packed_class_offset(plan, bits, cls, &off, nullptr);
    return launch_one(plan, cls, nullptr, bits, d_packed, d_scales, off, (cudaStream_t)stream);
}

eri_status_t eri_compute_compressed(eri_plan_t plan, int32_t bits, void *d_packed, float *d_scales,
                                    void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4)
        return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    size_t off = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        const int neri = class_neri(c);
        eri_status_t s = launch_one(plan, c, nullptr, bits, d_packed, d_scales, off, (cudaStream_t)stream);
        if (s != ERI_OK) return s;
        off += packed_segment_bytes(plan->count[c], neri, bits);
    }
    return ERI_OK;
}

eri_status_t eri_compute_compressed_to_host(eri_plan_t plan, int32_t bits, void *d_packed,
                                            float *d_scales, void *h_packed, float *h_scales,
                                            void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales || !h_packed || !h_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4)
        return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!plan->copy_stream) e = cudaStreamCreateWithFlags(&plan->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !plan->copy_done)
        e = cudaEventCreateWithFlags(&plan->copy_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e);
    size_t off = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        const size_t seg = packed_segment_bytes(plan->count[c], class_neri(c), bits);
        if (plan->count[c] > 0) {
            eri_status_t st = launch_one(plan, c, nullptr, bits, d_packed, d_scales, off, s);
            if (st != ERI_OK) return st;
            if (!plan->class_ev[c] &&
                (e = cudaEventCreateWithFlags(&plan->class_ev[c], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_status(e);
            // the class's codes and scales leave while the next classes compute (one copy stream:
            // more in flight measured no faster, the host link being the bound)
            e = cudaEventRecord(plan->class_ev[c], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->copy_stream, plan->class_ev[c], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(static_cast<char *>(h_packed) + off,
                                    static_cast<const char *>(d_packed) + off, seg,
                                    cudaMemcpyDeviceToHost, plan->copy_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_scales + plan->first[c], d_scales + plan->first[c],
                                    sizeof(float) * (size_t)plan->count[c], cudaMemcpyDeviceToHost,
                                    plan->copy_stream);
            if (e != cudaSuccess) return cuda_status(e);
        }
        off += seg;
    }
    // the caller's stream completes only after the last copy
    e = cudaEventRecord(plan->copy_done, plan->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->copy_done, 0);
    return cuda_status(e);
}

eri_status_t eri_backward(eri_plan_t plan, const double *d_G, double *d_dR, double *d_dalpha,
                          void *stream) {
    if (!plan || (plan->nq > 0 && !d_G) || (!d_dR && plan->n_shells > 0) ||
        (!d_dalpha && plan->n_prims > 0))
        return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_G) % 8 || reinterpret_cast<uintptr_t>(d_dR) % 8 ||
        reinterpret_cast<uintptr_t>(d_dalpha) % 8)
        return ERI_E_INVALID;
    // the adjoint of a class runs in that class's precision: FP64, or FP32 recurrences with FP64
    // geometry, roots and accumulation (the mixed adjoint)
    // (none for classes with a g shell)
    auto backward_of = [&](int c) -> BackwardFn {
        const int cc = canonicalise(c).cls;
        if (class_has_g(cc)) return nullptr;
        return class_precision(plan, c) == ERI_FP64 ? g_backward[cc] : g_backward_mixed[cc];
    };
    for (int c = 0; c < kNumClassIds; ++c)
        if (plan->count[c] > 0 && !backward_of(c)) return ERI_E_UNSUPPORTED;
    cudaSetDevice(plan->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_dR, 0, sizeof(double) * 3 * (size_t)plan->n_shells, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_dalpha, 0, sizeof(double) * (size_t)plan->n_prims, st);
    if (e != cudaSuccess) return cuda_status(e);
    ShellsDev sh{plan->d_cx, plan->d_cy, plan->d_cz, plan->d_pofs, plan->d_nprim, plan->d_exps, plan->d_cn};
    for (int c = 0; c < kNumClassIds; ++c) {
        if (plan->count[c] == 0) continue;
        Canon cn = canonicalise(c);
        ClassArgs a{};
        for (int k = 0; k < 4; ++k) {
            a.perm[k] = cn.perm[k];
            a.ostride[k] = cn.ostride[k];
        }
        a.quartets = plan->d_quartets + plan->first[c];
        a.nq = plan->count[c];
        a.err = plan->d_err;
        e = backward_of(c)(sh, plan->tables, a, d_G + plan->fp64_off[c], d_dR, d_dalpha, st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return ERI_OK;
}

eri_status_t eri_compute_compressed_batched(eri_plan_t plan, int32_t bits, void *d_packed,
                                            float *d_scales, void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4)
        return ERI_E_INVALID;
    if (plan->nq == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    eri_status_t st = ensure_batched_resources(plan);
    if (st != ERI_OK) return st;
    if (!plan->graph || plan->g_bits != bits || plan->g_prec != plan->precision ||
        plan->g_packed != d_packed || plan->g_scales != d_scales) {
        if (plan->graph) {
            cudaGraphExecDestroy(plan->graph);
            plan->graph = nullptr;
        }
        // capture the fork/launch/join sequence once on a side stream and keep the executable
        cudaStream_t origin = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(origin);
            return cuda_status(e);
        }
        st = enqueue_batched(plan, bits, d_packed, d_scales, origin);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(origin, &g);
        cudaStreamDestroy(origin);
        if (st != ERI_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaGraphInstantiate(&plan->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_status(e);
        plan->g_bits = bits;
        plan->g_prec = plan->precision;
        plan->g_packed = d_packed;
        plan->g_scales = d_scales;
    }
    return cuda_status(cudaGraphLaunch(plan->graph, (cudaStream_t)stream));
}

eri_status_t eri_compute_compressed_queue(eri_plan_t plan, int32_t bits, void *d_packed,
                                          float *d_scales, void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4)
        return ERI_E_INVALID;
    if (plan->nq == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = ensure_scratch(plan);
    const size_t table = queue_table_bytes();
    if (e == cudaSuccess && !plan->d_queue) e = cudaMalloc(&plan->d_queue, table + 16);
    if (e != cudaSuccess) return cuda_status(e);
    size_t total = 0;
    eri_output_bytes(plan, bits, &total, nullptr);
    // tiles OR their edge words into the output
    if ((e = cudaMemsetAsync(d_packed, 0, total, s)) != cudaSuccess) return cuda_status(e);
    std::vector<QueueSpec> spec;
    size_t off = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        if (plan->count[c] > 0) {
            QueueSpec q;
            class_ls(canonicalise(c).cls, q.L);
            q.a = class_args(plan, c, nullptr, bits, d_packed, d_scales, off);
            spec.push_back(q);
        }
        off += packed_segment_bytes(plan->count[c], class_neri(c), bits);
    }
    ShellsDev sh{plan->d_cx, plan->d_cy, plan->d_cz, plan->d_pofs, plan->d_nprim, plan->d_exps, plan->d_cn};
    e = launch_queue(sh, plan->tables, spec.data(), (int)spec.size(), plan->precision == ERI_MIXED, bits,
                     plan->d_err, plan->d_queue,
                     reinterpret_cast<unsigned long long *>(static_cast<char *>(plan->d_queue) + table),
                     static_cast<double *>(plan->d_setup), kScratchBytes, plan->device, s);
    return cuda_status(e);
}

eri_status_t eri_autotune(eri_plan_t plan, int32_t bits, void *d_packed, float *d_scales,
                          const char *cache_path, void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    eri_status_t st = ensure_batched_resources(plan);
    if (st != ERI_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, plan->device) != cudaSuccess) return ERI_E_CUDA;
    std::string gpu = prop.name;
    for (auto &ch : gpu)
        if (ch == ' ') ch = '_';
    // cached choices: lines "gpu variant bits canonical_class force_phase grid"
    std::vector<int> known(256 * kNumVariants, 0);
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "r")) {
            char name[256];
            int v, b, c, fp, gr;
            while (std::fscanf(f, "%255s %d %d %d %d %d", name, &v, &b, &c, &fp, &gr) == 6)
                if (gpu == name && v >= 0 && v < kNumVariants && b == bits && c >= 0 && c < 256) {
                    plan->tune_phase[c * kNumVariants + v] = fp;
                    plan->tune_grid[c * kNumVariants + v] = gr;
                    known[c * kNumVariants + v] = 1;
                }
            std::fclose(f);
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ShellsDev sh{plan->d_cx, plan->d_cy, plan->d_cz, plan->d_pofs, plan->d_nprim, plan->d_exps, plan->d_cn};
    std::vector<std::string> lines;
    size_t o = 0;
    std::vector<size_t> off(kNumClassIds);
    for (int c = 0; c < kNumClassIds; ++c) {
        off[c] = o;
        o += packed_segment_bytes(plan->count[c], class_neri(c), bits);
    }
    std::vector<int> done(256 * kNumVariants, 0);
    for (int c = 0; c < 256; ++c) {  // the run-time-L kernels of g classes have no choices
        if (plan->count[c] == 0) continue;
        int cc = canonicalise(c).cls;
        const int variant = class_variant(plan, c);
        if (known[cc * kNumVariants + variant] || done[cc * kNumVariants + variant]) continue;
        done[cc * kNumVariants + variant] = 1;
        LaunchFn fn = g_launch[cc * kNumVariants + variant];
        ClassArgs a = class_args(plan, c, nullptr, bits, d_packed, d_scales, off[c]);
        int cand_phase[2] = {0, 1};
        int n_phase = g_info[cc * kNumVariants + variant].tpq ? 2 : 1;
        int grids[3] = {0, prop.multiProcessorCount, 2 * prop.multiProcessorCount};
        float best = 1e30f;
        int bp = 0, bg = 0;
        for (int ip = 0; ip < n_phase; ++ip)
            for (int ig = 0; ig < 3; ++ig) {
                LaunchOpts lo;
                lo.device = plan->device;
                lo.counter = plan->d_counters + c;
                lo.force_phase = n_phase == 2 ? cand_phase[ip] : 0;
                lo.grid = grids[ig];
                float ms = 0.0f;
                for (int rep = 0; rep < 2; ++rep) {  // first run warms up
                    cudaMemsetAsync(plan->d_counters + c, 0, sizeof(unsigned long long), s);
                    cudaEventRecord(e0, s);
                    if (fn(sh, plan->tables, a, s, lo) != cudaSuccess) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return ERI_E_CUDA;
                    }
                    cudaEventRecord(e1, s);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                if (ms < best) {
                    best = ms;
                    bp = lo.force_phase;
                    bg = lo.grid;
                }
            }
        plan->tune_phase[cc * kNumVariants + variant] = bp;
        plan->tune_grid[cc * kNumVariants + variant] = bg;
        char buf[512];
        std::snprintf(buf, sizeof(buf), "%s %d %d %d %d %d\n", gpu.c_str(), variant, bits, cc, bp, bg);
        lines.push_back(buf);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path && !lines.empty()) {
        if (FILE *f = std::fopen(cache_path, "a")) {
            for (auto &l : lines) std::fputs(l.c_str(), f);
            std::fclose(f);
        }
    }
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    return cudaGetLastError() == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}

eri_status_t eri_plan_class_kernels(eri_plan_t plan, int32_t cls, char *buf, size_t len) {
    if (!plan || !class_id_valid(cls) || !buf || len == 0) return ERI_E_INVALID;
    buf[0] = 0;
    const int v = class_variant(plan, cls);
    const Canon c = canonicalise(cls);
    if (class_has_g(c.cls)) {
        const char *nm = generic_kernel_names(v != 0, true);
        if (std::strlen(nm) + 1 > len) return ERI_E_INVALID;
        std::memcpy(buf, nm, std::strlen(nm) + 1);
        return ERI_OK;
    }
    const int k = c.cls * kNumVariants + v;
    if (!g_launch[k]) return ERI_E_UNSUPPORTED;
    const bool split = plan->max_nprim == 1 && g_info[k].setup;
    const bool tpq = g_info[k].tpq && v != 2;
    char cfg[64];
    std::snprintf(cfg, sizeof(cfg), "Cfg<%d, %d, %d, %d, %s>", (c.cls >> 6) & 3, (c.cls >> 4) & 3,
                  (c.cls >> 2) & 3, c.cls & 3, v == 0 ? "double" : "float");
    // the launch choice of launch_class (eri_kernels.cuh) for a per-class call
    std::string name;
    if (tpq && split)
        name = std::string("eri_setup_kernel<") + cfg + "> + eri_tpq_kernel<" + cfg + ", 1>";
    else if (tpq)
        name = std::string("eri_tpq_kernel<") + cfg + ", 0>";
    else if (split)
        name = std::string("eri_setup_kernel<") + cfg + "> + eri_class_kernel<" + cfg + ", 0, 1>";
    else
        name = std::string("eri_class_kernel<") + cfg + (v == 2 ? ", 1, 0>" : ", 0, 0>");
    if (name.size() + 1 > len) return ERI_E_INVALID;
    std::memcpy(buf, name.c_str(), name.size() + 1);
    return ERI_OK;
}

eri_status_t eri_plan_class_launches(eri_plan_t plan, int32_t cls, int32_t *n_launches) {
    if (!plan || !class_id_valid(cls) || !n_launches) return ERI_E_INVALID;
    *n_launches = 0;
    if (plan->count[cls] == 0) return ERI_OK;
    const int v = class_variant(plan, cls);
    if (class_has_g(canonicalise(cls).cls)) {
        *n_launches = generic_launches(plan->count[cls], class_neri(cls), true, kScratchBytes);
        return ERI_OK;
    }
    const int k = canonicalise(cls).cls * kNumVariants + v;
    if (!g_launch[k]) return ERI_E_UNSUPPORTED;
    const bool split = plan->max_nprim == 1 && g_info[k].setup;
    *n_launches = split ? 2 * (int32_t)((plan->count[cls] + kSetupChunk - 1) / kSetupChunk) : 1;
    return ERI_OK;
}

eri_status_t eri_plan_calibrate_precision(eri_plan_t plan, int32_t bits, int64_t sample,
                                          float max_err_steps, void *stream) {
    if (!plan || bits < 2 || bits > 24 || sample < 1) return ERI_E_INVALID;
    if (!(max_err_steps > 0.0f && max_err_steps <= 1.0f)) return ERI_E_INVALID;
    if (plan->nq == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    size_t maxv = 0;
    for (int c = 0; c < kNumClassIds; ++c)
        maxv = std::max(maxv, (size_t)std::min<long long>(plan->count[c], sample) * class_neri(c));
    double *da = nullptr, *db = nullptr;
    unsigned int *dres = nullptr;
    cudaError_t e = cudaMalloc(&da, maxv * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&db, maxv * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dres, kNumClassIds * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(dres, 0, kNumClassIds * sizeof(unsigned int), s);
    for (int c = 0; e == cudaSuccess && c < kNumClassIds; ++c) {
        if (plan->count[c] == 0) continue;
        const long long n = std::min<long long>(plan->count[c], sample);
        const int neri = class_neri(c);
        double *bufs[2] = {da, db};
        for (int k = 0; k < 2; ++k) {
            ClassArgs a = class_args(plan, c, bufs[k], 0, nullptr, nullptr, 0);
            a.nq = n;
            a.out_fp64 = bufs[k];
            const int variant = k == 0 ? 0 : (plan->max_nprim > 1 ? 2 : 1);
            eri_status_t st = launch_class_args(plan, c, a, variant, s);
            if (st != ERI_OK) {
                cudaFree(da);
                cudaFree(db);
                cudaFree(dres);
                return st;
            }
        }
        if (e == cudaSuccess) {
            calib_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(da, db, n, neri, dres + c);
            e = cudaGetLastError();
        }
    }
    std::vector<unsigned int> res(kNumClassIds, 0u);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res.data(), dres, kNumClassIds * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dres);
    if (e != cudaSuccess) return cuda_status(e);
    // a class keeps the FP32 recurrences when its measured error stays below max_err_steps
    // quantisation steps, one step being eps / b_max = 1 / (2^{bits-1} - 1)
    const float thr = max_err_steps / (float)((1u << (bits - 1)) - 1u);
    for (int c = 0; c < kNumClassIds; ++c) {
        if (plan->count[c] == 0) continue;
        float err;
        std::memcpy(&err, &res[c], sizeof(float));
        plan->class_err[c] = err;
        plan->class_prec[c] = err < thr ? ERI_MIXED : ERI_FP64;
    }
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    return ERI_OK;
}

eri_status_t eri_plan_screening(eri_plan_t plan, int64_t *candidates, int64_t *kept) {
    if (!plan) return ERI_E_INVALID;
    if (candidates) *candidates = plan->screen_candidates;
    if (kept) *kept = plan->screen_kept;
    return ERI_OK;
}

eri_status_t eri_plan_quartets(eri_plan_t plan, int32_t *quartets_out) {
    if (!plan || (!quartets_out && plan->nq > 0)) return ERI_E_INVALID;
    if (plan->nq == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    return cuda_status(cudaMemcpy(quartets_out, plan->d_quartets, plan->nq * sizeof(int4), cudaMemcpyDeviceToHost));
}

eri_status_t eri_plan_num_basis_functions(eri_plan_t plan, int64_t *n_bf) {
    if (!plan || !n_bf) return ERI_E_INVALID;
    *n_bf = plan->n_bf;
    return ERI_OK;
}

eri_status_t eri_digest_jk(eri_plan_t plan, int32_t bits, const void *d_packed, const float *d_scales,
                           const double *d_D, double *d_J, double *d_K, int32_t flags, void *stream) {
    if (!plan || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (flags & ~(ERI_DIGEST_UNIQUE8 | ERI_DIGEST_ACCUMULATE | ERI_DIGEST_SYMMETRIC)) return ERI_E_INVALID;
    const bool sym = (flags & ERI_DIGEST_SYMMETRIC) != 0;
    if (sym && !(flags & ERI_DIGEST_UNIQUE8)) return ERI_E_INVALID;
    if (plan->n_bf > 0 && (!d_D || !d_J || !d_K)) return ERI_E_INVALID;
    if (plan->nq > 0 && (!d_packed || !d_scales)) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_packed) % 4 || reinterpret_cast<uintptr_t>(d_scales) % 4 ||
        reinterpret_cast<uintptr_t>(d_D) % 8 || reinterpret_cast<uintptr_t>(d_J) % 8 ||
        reinterpret_cast<uintptr_t>(d_K) % 8)
        return ERI_E_INVALID;
    for (int c = 256; c < kNumClassIds; ++c)
        if (plan->count[c] > 0) return ERI_E_UNSUPPORTED;  // classes with a g shell
    if (plan->n_bf == 0) return ERI_OK;
    cudaSetDevice(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    const long long n2 = plan->n_bf * plan->n_bf;
    cudaError_t e = cudaSuccess;
    if (!(flags & ERI_DIGEST_ACCUMULATE)) {
        e = cudaMemsetAsync(d_J, 0, sizeof(double) * (size_t)n2, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_K, 0, sizeof(double) * (size_t)n2, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (plan->nq == 0) return ERI_OK;
    if (!plan->d_D32 && (e = cudaMalloc(&plan->d_D32, sizeof(float) * (size_t)n2)) != cudaSuccess)
        return cuda_status(e);
    if (!plan->d_digest && (e = cudaMalloc(&plan->d_digest, digest_table_bytes())) != cudaSuccess)
        return cuda_status(e);
    if ((e = digest_density_f32(d_D, n2, plan->d_D32, s)) != cudaSuccess) return cuda_status(e);
    std::vector<DigestClass> dcs;
    size_t off = 0;
    for (int c = 0; c < kNumClassIds; ++c) {
        const size_t seg = packed_segment_bytes(plan->count[c], class_neri(c), bits);
        if (plan->count[c] > 0) {
            DigestClass dc;
            dc.cls = c;
            dc.quartets = plan->d_quartets + plan->first[c];
            dc.nq = plan->count[c];
            dc.packed = reinterpret_cast<const uint32_t *>(static_cast<const char *>(d_packed) + off);
            dc.scales = d_scales + plan->first[c];
            dcs.push_back(dc);
        }
        off += seg;
    }
    e = digest_all(dcs.data(), (int)dcs.size(), bits, (flags & ERI_DIGEST_UNIQUE8) != 0, sym, plan->d_bfoff,
                   plan->d_D32, plan->n_bf, d_J, d_K, plan->d_digest, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (sym) {
        if ((e = digest_symmetrise(d_J, plan->n_bf, s)) != cudaSuccess) return cuda_status(e);
        if ((e = digest_symmetrise(d_K, plan->n_bf, s)) != cudaSuccess) return cuda_status(e);
    }
    return ERI_OK;
}

eri_status_t eri_sync(eri_plan_t plan, void *stream) {
    if (!plan) return ERI_E_INVALID;
    cudaSetDevice(plan->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return ERI_E_CUDA;
    int err = 0;
    e = cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ERI_E_CUDA;
    if (err) cudaMemset(plan->d_err, 0, sizeof(int));
    if (err & 1) return ERI_E_NUMERIC;
    return ERI_OK;
}

}  // extern "C"
