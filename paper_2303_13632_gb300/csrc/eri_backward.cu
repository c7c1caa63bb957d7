// eri_backward.cu -- instantiates the adjoint kernels of the canonical classes with every
// angular momentum <= 2 (s, p, d; the extended index ranges of f shells exceed the
// per-CTA shared memory in FP64) and registers their launchers.
#include "eri_backward.cuh"
#include "eri_internal.h"

namespace eri {

template <int IDX>
struct RegisterBackward {
    static void apply(BackwardFn *table) {
        if constexpr (IDX < kNumCanonical) {
            constexpr int cls = canonical_class(IDX);
            constexpr int La = (cls >> 6) & 3, Lb = (cls >> 4) & 3, Lc = (cls >> 2) & 3, Ld = cls & 3;
            if constexpr (La <= 2 && Lb <= 2 && Lc <= 2 && Ld <= 2)
                table[cls] = &launch_backward<La, Lb, Lc, Ld>;
            RegisterBackward<IDX + 1>::apply(table);
        }
    }
};

void eri_register_backward(BackwardFn *table) { RegisterBackward<0>::apply(table); }

}  // namespace eri
