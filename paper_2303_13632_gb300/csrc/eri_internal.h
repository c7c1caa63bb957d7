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
