// eri_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "../../include/eri.h"
#include "eri_device.cuh"

namespace eri {

// Device addresses of the constant tables on the current device (uploaded on first use).
cudaError_t tables_for_current_device(Tables *out);

// Launcher of one canonical class kernel in one arithmetic variant.
using LaunchFn = cudaError_t (*)(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                                 cudaStream_t stream);
// Variants: 0 = FP64, 1 = mixed, 2 = mixed with Kahan-compensated primitive sums.
constexpr int kNumVariants = 3;

// Launcher of one canonical class's adjoint kernel (FP64).
using BackwardFn = cudaError_t (*)(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                                   const double *G, double *dR, double *dalpha, cudaStream_t stream);
void eri_register_backward(BackwardFn *table);

// Each class translation unit fills table[cls * kNumVariants + variant] for its classes.
constexpr int kNumTU = 16;
#define ERI_DECLARE_REGISTER(K) void eri_register_tu_##K(LaunchFn *table);
ERI_DECLARE_REGISTER(0) ERI_DECLARE_REGISTER(1) ERI_DECLARE_REGISTER(2) ERI_DECLARE_REGISTER(3)
ERI_DECLARE_REGISTER(4) ERI_DECLARE_REGISTER(5) ERI_DECLARE_REGISTER(6) ERI_DECLARE_REGISTER(7)
ERI_DECLARE_REGISTER(8) ERI_DECLARE_REGISTER(9) ERI_DECLARE_REGISTER(10) ERI_DECLARE_REGISTER(11)
ERI_DECLARE_REGISTER(12) ERI_DECLARE_REGISTER(13) ERI_DECLARE_REGISTER(14) ERI_DECLARE_REGISTER(15)
#undef ERI_DECLARE_REGISTER

}  // namespace eri
