// eri_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/eri.h"
#include "eri_device.cuh"

namespace eri {

// Device addresses of the constant tables on the current device (uploaded on first use).
cudaError_t tables_for_current_device(Tables *out);

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
void eri_register_backward(BackwardFn *table);

// Each class translation unit fills table[cls * kNumVariants + variant] for its classes.
constexpr int kNumTU = 16;
// info[cls * kNumVariants + v] describes that launcher.
struct KernelInfo {
    bool tpq;    // has a thread-per-quartet kernel (LaunchOpts::force_phase selects the other)
    bool setup;  // primitive (K = 1) plans run it through the setup kernel: the caller passes
                 // LaunchOpts::scratch and at most kSetupChunk quartets per launch
};
#define ERI_DECLARE_REGISTER(K) void eri_register_tu_##K(LaunchFn *table, KernelInfo *info);
ERI_DECLARE_REGISTER(0) ERI_DECLARE_REGISTER(1) ERI_DECLARE_REGISTER(2) ERI_DECLARE_REGISTER(3)
ERI_DECLARE_REGISTER(4) ERI_DECLARE_REGISTER(5) ERI_DECLARE_REGISTER(6) ERI_DECLARE_REGISTER(7)
ERI_DECLARE_REGISTER(8) ERI_DECLARE_REGISTER(9) ERI_DECLARE_REGISTER(10) ERI_DECLARE_REGISTER(11)
ERI_DECLARE_REGISTER(12) ERI_DECLARE_REGISTER(13) ERI_DECLARE_REGISTER(14) ERI_DECLARE_REGISTER(15)
#undef ERI_DECLARE_REGISTER

}  // namespace eri
