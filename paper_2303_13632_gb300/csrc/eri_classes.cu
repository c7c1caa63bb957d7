// eri_classes.cu -- instantiates the kernels of the canonical classes whose index is
// congruent to ERI_TU modulo kNumTU, in the three arithmetic variants.  Compiled once per
// unit with -DERI_TU=<0..15> so the 55 canonical classes build in parallel.
#include "eri_internal.h"
#include "eri_kernels.cuh"

#ifndef ERI_TU
#error "compile with -DERI_TU=<0..15>"
#endif

#define ERI_CAT2(a, b) a##b
#define ERI_CAT(a, b) ERI_CAT2(a, b)
#define ERI_REGISTER_NAME ERI_CAT(eri_register_tu_, ERI_TU)

namespace eri {

template <int IDX>
struct Register {
    static void apply(LaunchFn *table, KernelInfo *info) {
        if constexpr (IDX < kNumCanonical) {
            if constexpr (IDX % kNumTU == ERI_TU) {
                constexpr int cls = canonical_class(IDX);
                constexpr int La = (cls >> 6) & 3, Lb = (cls >> 4) & 3, Lc = (cls >> 2) & 3,
                              Ld = cls & 3;
                table[cls * kNumVariants + 0] = &launch_class<La, Lb, Lc, Ld, double, false>;
                table[cls * kNumVariants + 1] = &launch_class<La, Lb, Lc, Ld, float, false>;
                table[cls * kNumVariants + 2] = &launch_class<La, Lb, Lc, Ld, float, true>;
                info[cls * kNumVariants + 0] = {Cfg<La, Lb, Lc, Ld, double>::TPQ,
                                                 Cfg<La, Lb, Lc, Ld, double>::USES_SETUP};
                info[cls * kNumVariants + 1] = {Cfg<La, Lb, Lc, Ld, float>::TPQ,
                                                 Cfg<La, Lb, Lc, Ld, float>::USES_SETUP};
                info[cls * kNumVariants + 2] = {false, false};  // contracted: fused kernels
                // setup records fit the setup buffer (kSetupFieldsMax doubles per quartet)
                static_assert(Cfg<La, Lb, Lc, Ld, double>::SETUP_FIELDS <= kSetupFieldsMax, "setup");
                static_assert(Cfg<La, Lb, Lc, Ld, float>::SETUP_FIELDS * sizeof(float) <=
                                  kSetupFieldsMax * sizeof(double), "setup");
            }
            Register<IDX + 1>::apply(table, info);
        }
    }
};

void ERI_REGISTER_NAME(LaunchFn *table, KernelInfo *info) { Register<0>::apply(table, info); }

}  // namespace eri
