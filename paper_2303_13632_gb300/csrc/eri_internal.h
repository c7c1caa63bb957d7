// eri_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/eri.h"
#include "eri_device.cuh"

namespace eri {

// Device addresses of the constant tables on the current device (uploaded on first use).
cudaError_t tables_for_current_device(Tables *out);
// FP32 copies of the table parts the mixed-precision setup reads (eri_tables.cu).
void mixed_table_copies(std::vector<float> &tail_m, std::vector<float> &t01_f);

// Class ids.  Classes without a g shell keep the ids of the 256 classes of Sec. III-A,
// ((La*4 + Lb)*4 + Lc)*4 + Ld; classes with a g shell (L = 4) take 256 + ((La*5 + Lb)*5 + Lc)*5
// + Ld.  The slots 256 + ... whose four angular momenta are all <= 3 are never used, so a plan's
// per-class arrays have kNumClassIds entries of which 625 can be non-empty.
constexpr int kLmax = 4;
constexpr int kNumClassIds = 256 + 625;
__host__ __device__ inline int class_id_of(int La, int Lb, int Lc, int Ld) {
    if (La < 4 && Lb < 4 && Lc < 4 && Ld < 4) return ((La * 4 + Lb) * 4 + Lc) * 4 + Ld;
    return 256 + ((La * 5 + Lb) * 5 + Lc) * 5 + Ld;
}
__host__ __device__ inline void class_ls(int cls, int L[4]) {
    if (cls < 256) {
        L[0] = (cls >> 6) & 3; L[1] = (cls >> 4) & 3; L[2] = (cls >> 2) & 3; L[3] = cls & 3;
    } else {
        int r = cls - 256;
        L[3] = r % 5; r /= 5;
        L[2] = r % 5; r /= 5;
        L[1] = r % 5; L[0] = r / 5;
    }
}
// true for the ids of actual classes (0..255 and the slots with a g shell)
inline bool class_id_valid(int cls) {
    if (cls < 0 || cls >= kNumClassIds) return false;
    if (cls < 256) return true;
    int L[4];
    class_ls(cls, L);
    return L[0] == 4 || L[1] == 4 || L[2] == 4 || L[3] == 4;
}
inline bool class_has_g(int cls) { return cls >= 256; }

// Classes with a g shell run one kernel whose angular momenta are run-time values
// (eri_generic.cu): L = the canonical angular momenta, a the canonical class's arguments (its
// quartets, permutation, output strides and output).  FP64 output is written to a.out_fp64;
// compressed output goes through `scratch` (scratch_bytes of device memory, FP64 values of up to
// scratch_bytes / (8 n_ERIQ) quartets at a time).  mixed: FP32 recurrences and quadrature from
// FP64 setup values, FP64 sums over primitives.
cudaError_t launch_generic(const ShellsDev &sh, const Tables &tb, const ClassArgs &a, const int L[4],
                           bool mixed, double *scratch, size_t scratch_bytes, cudaStream_t stream);
// launches launch_generic makes for nq quartets of n_ERIQ = neri, and the kernel names
int generic_launches(long long nq, int neri, bool compressed, size_t scratch_bytes);
const char *generic_kernel_names(bool mixed, bool compressed);

// One persistent launch of the run-time-L kernel over every class of a plan from one work queue
// of tiles, compressing each tile in the same launch (eri_generic.cu).  classes[i]: the canonical
// angular momenta and the arguments of one non-empty class (compressed output; the packed output
// must be zero before the launch).  d_table: queue_table_bytes() of device memory, d_counter one
// device word, scratch: FP64 values of one tile per resident CTA.
struct QueueSpec {
    int L[4];
    ClassArgs a;
};
size_t queue_table_bytes();
cudaError_t launch_queue(const ShellsDev &sh, const Tables &tb, const QueueSpec *classes, int n_classes,
                         bool mixed, int bits, int *err, void *d_table, unsigned long long *d_counter,
                         double *scratch, size_t scratch_bytes, int device, cudaStream_t stream);

// Quartets per launch of the split setup/recurrence path (a multiple of 32 so that every chunk
// starts on a 32-bit word of the packed stream) and the widest setup record (n_Rys = 7).
constexpr long long kSetupChunk = 1LL << 20;
constexpr int kSetupFieldsMax = 8 + 7 * 10;
// largest primitive-pair table a plan builds (bytes); larger plans compute the pair
// quantities per quartet instead
constexpr double kPairTableMaxBytes = 16.0 * 1024 * 1024 * 1024;

// Launcher of one canonical class kernel in one arithmetic variant.
using LaunchFn = cudaError_t (*)(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                                 cudaStream_t stream, const LaunchOpts &opts);
// Variants: 0 = FP64, 1 = mixed, 2 = mixed with Kahan-compensated primitive sums.
constexpr int kNumVariants = 3;

// Launcher of one canonical class's adjoint kernel (FP64).
using BackwardFn = cudaError_t (*)(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                                   const double *G, double *dR, double *dalpha, cudaStream_t stream);
// Each adjoint unit fills the FP64 and the mixed-precision table for its classes.
void eri_register_backward_0(BackwardFn *table, BackwardFn *table_mixed);
void eri_register_backward_1(BackwardFn *table, BackwardFn *table_mixed);
void eri_register_backward_2(BackwardFn *table, BackwardFn *table_mixed);
void eri_register_backward_3(BackwardFn *table, BackwardFn *table_mixed);

// Each class translation unit fills table[cls * kNumVariants + variant] for its classes.
constexpr int kNumTU = 16;
// info[cls * kNumVariants + v] describes that launcher.
struct KernelInfo {
    bool tpq;    // has a thread-per-quartet kernel (LaunchOpts::force_phase selects the other)
    bool setup;  // primitive (K = 1) plans run it through the setup kernel: the caller passes
                 // LaunchOpts::scratch and at most kSetupChunk quartets per launch
};
// One class of a plan's compressed output, as the Coulomb/exchange digestion reads it.
struct DigestClass {
    int cls;               // generic class id
    const int4 *quartets;  // class-sorted shell ids (the caller's orientation)
    long long nq;
    const uint32_t *packed;  // first word of the class segment
    const float *scales;     // eps of the class's first quartet
};
// D (FP64, n values) rounded to FP32 into out.
cudaError_t digest_density_f32(const double *D, long long n, float *out, cudaStream_t stream);
// Bytes of the device table digest_all needs (per-class parameters and tile offsets).
size_t digest_table_bytes();
// Adds the contributions of the n_classes classes to J and K in one launch (see eri_digest.cu);
// with `symmetric` (D symmetric) each item adds to one of its two transposed destinations, and
// digest_symmetrise finishes.  d_table: digest_table_bytes() of device memory, written on `stream`.
cudaError_t digest_all(const DigestClass *classes, int n_classes, int bits, bool unique8, bool symmetric,
                       const int *bfoff, const float *D32, long long nbf, double *J, double *K,
                       void *d_table, cudaStream_t stream);
// M = (M + M^T) / 2 (n x n, row major).
cudaError_t digest_symmetrise(double *M, long long n, cudaStream_t stream);

// Device quartet lists (eri_screen.cu).  Diagonal quartets (i j | i j) of every unordered pair
// P = i (i + 1) / 2 + j, i >= j.
cudaError_t screen_diag_quartets(long long npairs, int4 *out, cudaStream_t s);
// out[q] = sqrt(max_v |x[q * neri + v]|) for n quartets.
cudaError_t screen_absmax_sqrt(const double *x, long long n, int neri, double *out, cudaStream_t s);
// out[idx[i]] = v[i].
cudaError_t screen_scatter(const double *v, const int *idx, long long n, double *out, cudaStream_t s);
// The 8-fold unique quartets of the pairs with factors d_Q (see eri_screen.cu), screened at tau
// (tau = 0: none), shard sidx of scount; allocates *d_out (n_out quartets); *total = the count
// before sharding; cudaErrorNotSupported if more than max_out quartets would be kept.
// Synchronous on s.
cudaError_t screen_unique8(const double *d_Q, long long npairs, double tau, long long sidx,
                           long long scount, int4 **d_out, long long *n_out, long long *total,
                           long long max_out, cudaStream_t s);
// Keeps the quartets of d_in with Q_ij Q_kl >= tau, in order; allocates *d_out and *d_idx (the
// input index of every kept quartet).  Synchronous on s.
cudaError_t screen_filter(const int4 *d_in, long long n, const double *d_Q, double tau, int4 **d_out,
                          int **d_idx, long long *n_out, cudaStream_t s);

#define ERI_DECLARE_REGISTER(K) void eri_register_tu_##K(LaunchFn *table, KernelInfo *info);
ERI_DECLARE_REGISTER(0) ERI_DECLARE_REGISTER(1) ERI_DECLARE_REGISTER(2) ERI_DECLARE_REGISTER(3)
ERI_DECLARE_REGISTER(4) ERI_DECLARE_REGISTER(5) ERI_DECLARE_REGISTER(6) ERI_DECLARE_REGISTER(7)
ERI_DECLARE_REGISTER(8) ERI_DECLARE_REGISTER(9) ERI_DECLARE_REGISTER(10) ERI_DECLARE_REGISTER(11)
ERI_DECLARE_REGISTER(12) ERI_DECLARE_REGISTER(13) ERI_DECLARE_REGISTER(14) ERI_DECLARE_REGISTER(15)
#undef ERI_DECLARE_REGISTER

}  // namespace eri
