// eri_noalloc.cu -- eri_compute_class_noalloc: ERIs of one class (FP64 or mixed) without any device
// allocation by this library.
//
// Some callers cannot let a library call cudaMalloc: applications that reserve all device
// memory up front and hand it out from their own pool (a late cudaMalloc would fail or break
// their accounting), and code whose latency budget rules out the implicit synchronisation
// cudaMalloc/cudaFree may cause.  The plan API allocates its device copies and a setup
// buffer; this entry point instead takes every input and output as caller-owned device
// memory and keeps its only scratch (the per-quartet setup buffer of the split
// setup/recurrence path) in a file-scope __device__ array, with the Rys and Boys tables in
// __device__ arrays initialised when the module loads.
#include <mutex>

#include "eri_internal.h"

namespace eri {

// Host copies of the tables (only the small index arrays are used on the host).
namespace host_tables {
#include "eri_tables.inc"
}  // namespace host_tables

// Device copies of the same tables: the generated arrays re-declared as __device__ data.
namespace device_tables {
#define static static __device__
#include "eri_tables.inc"
#undef static
}  // namespace device_tables

namespace {

// Setup buffer: the widest setup record for ERI_NOALLOC_MAX_QUARTETS quartets (about 10 MB,
// held by every GPU that loads the library until the process exits).
static __device__ __align__(256) double g_noalloc_scratch[(size_t)ERI_NOALLOC_MAX_QUARTETS *
                                                          kSetupFieldsMax];
// FP32 copies of table parts read by the mixed-precision setup, written once per device at
// set-up from host memory (a copy into these arrays, no allocation)
static __device__ float g_rys_tail_m[(RYS_POLY_LEN / (RYS_DEG + 1)) * (RYS_DEG + 1 - kRysTailMixed)];
static __device__ float g_boys_t01_f[BOYS_T01_LEN];

struct DeviceState {
    bool ready = false;
    Tables tables{};
    void *scratch = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
DeviceState g_state[kMaxDevices];
LaunchFn g_table[256 * kNumVariants];
KernelInfo g_info_unused[256 * kNumVariants];
std::once_flag g_table_once;

void fill_table() {
    eri_register_tu_0(g_table, g_info_unused); eri_register_tu_1(g_table, g_info_unused);
    eri_register_tu_2(g_table, g_info_unused); eri_register_tu_3(g_table, g_info_unused);
    eri_register_tu_4(g_table, g_info_unused); eri_register_tu_5(g_table, g_info_unused);
    eri_register_tu_6(g_table, g_info_unused); eri_register_tu_7(g_table, g_info_unused);
    eri_register_tu_8(g_table, g_info_unused); eri_register_tu_9(g_table, g_info_unused);
    eri_register_tu_10(g_table, g_info_unused); eri_register_tu_11(g_table, g_info_unused);
    eri_register_tu_12(g_table, g_info_unused); eri_register_tu_13(g_table, g_info_unused);
    eri_register_tu_14(g_table, g_info_unused); eri_register_tu_15(g_table, g_info_unused);
}

// Device addresses of the __device__ arrays for the current device (host code sees only a
// host-side stand-in under these names, so the addresses must come from the runtime).
cudaError_t device_state(DeviceState **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceState &s = g_state[dev];
    if (!s.ready) {
        void *p = nullptr;
        Tables t{};
        if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
        s.scratch = p;
        if ((e = cudaGetSymbolAddress(&p, device_tables::rys_poly_h)) != cudaSuccess) return e;
        t.rys_poly = static_cast<const double *>(p);
        if ((e = cudaGetSymbolAddress(&p, device_tables::rys_herm_x2_h)) != cudaSuccess) return e;
        t.herm_x2 = static_cast<const double *>(p);
        if ((e = cudaGetSymbolAddress(&p, device_tables::rys_herm_w_h)) != cudaSuccess) return e;
        t.herm_w = static_cast<const double *>(p);
        if ((e = cudaGetSymbolAddress(&p, device_tables::boys_grid_h)) != cudaSuccess) return e;
        t.boys_grid = static_cast<const double *>(p);
        if ((e = cudaGetSymbolAddress(&p, device_tables::boys_t01_h)) != cudaSuccess) return e;
        t.boys_t01 = static_cast<const double *>(p);
        if ((e = cudaGetSymbolAddress(&p, device_tables::rys_tail_f_h)) != cudaSuccess) return e;
        t.rys_tail = static_cast<const float *>(p);
        std::vector<float> tail_m, t01_f;
        mixed_table_copies(tail_m, t01_f);
        if (tail_m.size() * sizeof(float) != sizeof(g_rys_tail_m) || t01_f.size() * sizeof(float) != sizeof(g_boys_t01_f))
            return cudaErrorInvalidValue;
        if ((e = cudaGetSymbolAddress(&p, g_rys_tail_m)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(p, tail_m.data(), sizeof(g_rys_tail_m), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        t.rys_tail_m = static_cast<const float *>(p);
        if ((e = cudaGetSymbolAddress(&p, g_boys_t01_f)) != cudaSuccess) return e;
        if ((e = cudaMemcpy(p, t01_f.data(), sizeof(g_boys_t01_f), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        t.boys_t01_f = static_cast<const float *>(p);
        for (int i = 0; i <= kRysNmax; ++i) {
            t.tasym[i] = host_tables::rys_tasym_h[i];
            t.offset[i] = host_tables::rys_offset_h[i];
        }
        for (int i = 0; i <= kRysNmax + 1; ++i) t.herm_off[i] = host_tables::rys_herm_offset_h[i];
        s.tables = t;
        s.ready = true;
    }
    *out = &s;
    return cudaSuccess;
}

int nc(int L) { return (L + 1) * (L + 2) / 2; }

// Canonical representative of a generic class and the shell permutation / output strides
// (the same rule as the plan: larger L first within each pair, the pair with more
// components as the bra).
void canonical(int cls, int *perm, int *ostride, int *ccls) {
    int L[4] = {(cls >> 6) & 3, (cls >> 4) & 3, (cls >> 2) & 3, cls & 3};
    int bra[2] = {0, 1}, ket[2] = {2, 3};
    if (L[0] < L[1]) { bra[0] = 1; bra[1] = 0; }
    if (L[2] < L[3]) { ket[0] = 3; ket[1] = 2; }
    int p[4] = {bra[0], bra[1], ket[0], ket[1]};
    if (nc(L[bra[0]]) * nc(L[bra[1]]) < nc(L[ket[0]]) * nc(L[ket[1]])) {
        p[0] = ket[0]; p[1] = ket[1]; p[2] = bra[0]; p[3] = bra[1];
    }
    int g[4];
    g[3] = 1;
    for (int k = 2; k >= 0; --k) g[k] = g[k + 1] * nc(L[k + 1]);
    for (int k = 0; k < 4; ++k) {
        perm[k] = p[k];
        ostride[k] = g[p[k]];
    }
    *ccls = ((L[p[0]] * 4 + L[p[1]]) * 4 + L[p[2]]) * 4 + L[p[3]];
}

// Flags (bit 2 of *err) quartets whose shells are contracted: the split path computes one
// primitive quartet per quartet.
__global__ void noalloc_check_kernel(const int4 *__restrict__ q, long long n,
                                     const int *__restrict__ nprim, int *err) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int4 t = q[i];
    if (nprim[t.x] != 1 || nprim[t.y] != 1 || nprim[t.z] != 1 || nprim[t.w] != 1) atomicOr(err, 4);
}

}  // namespace

}  // namespace eri

using namespace eri;

extern "C" eri_status_t eri_compute_class_noalloc(int32_t cls, int32_t precision, const double *d_cx,
                                                  const double *d_cy, const double *d_cz,
                                                  const int32_t *d_pofs, const int32_t *d_nprim,
                                                  const double *d_exps, const double *d_cn,
                                                  const int32_t *d_quartets, int64_t n_quartets,
                                                  double *d_out, int32_t *d_err, void *stream) {
    if (class_id_valid(cls) && class_has_g(cls)) return ERI_E_UNSUPPORTED;  // L <= 3 only
    if (cls < 0 || cls > 255 || (precision != ERI_FP64 && precision != ERI_MIXED)) return ERI_E_INVALID;
    if (n_quartets < 0 || n_quartets > ERI_NOALLOC_MAX_QUARTETS) return ERI_E_INVALID;
    if (!d_err) return ERI_E_INVALID;
    if (n_quartets == 0) return ERI_OK;
    if (!d_cx || !d_cy || !d_cz || !d_pofs || !d_nprim || !d_exps || !d_cn || !d_quartets || !d_out)
        return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_quartets) % 16 || reinterpret_cast<uintptr_t>(d_out) % 8)
        return ERI_E_INVALID;
    std::call_once(g_table_once, fill_table);
    DeviceState *st = nullptr;
    if (device_state(&st) != cudaSuccess) return ERI_E_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ERI_E_CUDA;
    ClassArgs a{};
    int ccls = 0;
    canonical(cls, a.perm, a.ostride, &ccls);
    a.quartets = reinterpret_cast<const int4 *>(d_quartets);
    a.nq = n_quartets;
    a.out_fp64 = d_out;
    a.err = d_err;
    const int variant = precision == ERI_FP64 ? 0 : 1;
    LaunchFn fn = g_table[ccls * kNumVariants + variant];
    if (!fn) return ERI_E_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    noalloc_check_kernel<<<(unsigned)((n_quartets + 255) / 256), 256, 0, s>>>(a.quartets, n_quartets,
                                                                            d_nprim, d_err);
    if (cudaGetLastError() != cudaSuccess) return ERI_E_CUDA;
    ShellsDev sh{d_cx, d_cy, d_cz, d_pofs, d_nprim, d_exps, d_cn};
    LaunchOpts o;
    o.device = dev;
    o.scratch = st->scratch;
    return fn(sh, st->tables, a, s, o) == cudaSuccess ? ERI_OK : ERI_E_CUDA;
}
