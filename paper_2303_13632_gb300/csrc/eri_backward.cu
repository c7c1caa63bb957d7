// eri_backward.cu -- instantiates the adjoint kernels of the canonical classes whose index is
// congruent to ERI_BTU modulo 4 (compiled once per unit with -DERI_BTU=<0..3>) and registers
// their launchers: FP64 for classes with every angular momentum <= 2 (the extended index ranges
// of f shells exceed the per-CTA shared memory in FP64), FP32 recurrences (the mixed adjoint)
// for every class.
#include "eri_backward.cuh"
#include "eri_internal.h"

#ifndef ERI_BTU
#error "compile with -DERI_BTU=<0..3>"
#endif

#define ERI_BCAT2(a, b) a##b
#define ERI_BCAT(a, b) ERI_BCAT2(a, b)

namespace eri {

template <int IDX>
struct RegisterBackward {
    static void apply(BackwardFn *table, BackwardFn *table_mixed) {
        if constexpr (IDX < kNumCanonical) {
            if constexpr (IDX % 4 == ERI_BTU) {
                constexpr int cls = canonical_class(IDX);
                constexpr int La = (cls >> 6) & 3, Lb = (cls >> 4) & 3, Lc = (cls >> 2) & 3, Ld = cls & 3;
                if constexpr (La <= 2 && Lb <= 2 && Lc <= 2 && Ld <= 2)
                    table[cls] = &launch_backward<La, Lb, Lc, Ld, double>;
                table_mixed[cls] = &launch_backward<La, Lb, Lc, Ld, float>;
            }
            RegisterBackward<IDX + 1>::apply(table, table_mixed);
        }
    }
};

void ERI_BCAT(eri_register_backward_, ERI_BTU)(BackwardFn *table, BackwardFn *table_mixed) {
    RegisterBackward<0>::apply(table, table_mixed);
}

}  // namespace eri
