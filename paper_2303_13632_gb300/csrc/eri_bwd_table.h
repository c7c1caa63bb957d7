// eri_bwd_table.h -- index table of the adjoint's grouped contraction (plain C++17, evaluated at
// compile time; eri_backward.cuh places one per canonical class in device memory).
//
// The adjoint contracts G with the 2-D integrals axis by axis: for axis x and the x-components
// w = (i0, i1, i2, i3) of the four centres, W = sum of G I_y I_z over the outputs sharing them
// (y, z the axes after x in cyclic order).  The table lists, for each axis, the outputs group by
// group: entries start[w] .. start[w + 1] - 1 of e[x * N ..] belong to w (groups in the order
// w = ((i0 * (B + 1) + i1) * (Cc + 1) + i2) * (D + 1) + i3).  Each entry holds the output's
// canonical index ((ia * NB + ib) * NC + ic) * ND + id (bits 0-15), the offset of its
// y-components (bits 16-31) and of its z-components (bits 32-47) inside one (axis, root) block of
// the 2-D integrals on the index ranges extended by two, layout [a][c][b][d] with the (b, d)
// blocks padded to an odd length JLP.
#pragma once

namespace eri {

constexpr int bwd_ncart(int L) { return (L + 1) * (L + 2) / 2; }

template <int A, int B, int Cc, int D>
struct BwdTab {
    static constexpr int W1 = A + 1, W2 = B + 1, W3 = Cc + 1, W4 = D + 1, WN = W1 * W2 * W3 * W4;
    static constexpr int NB = bwd_ncart(B), NC = bwd_ncart(Cc), ND = bwd_ncart(D),
                         N = bwd_ncart(A) * NB * NC * ND;
    // extended index ranges (L + 2) of the 2-D integrals, as in GCfg
    static constexpr int LC1 = Cc + 3, LD1 = D + 3, JL = (B + 3) * (D + 3), JLP = JL % 2 ? JL : JL + 1;
    unsigned short start[WN + 1];
    unsigned long long e[3 * N];
};

// Cartesian index of the component with c0 along axis 0 and c1 along axis 1 (first component
// descending, then the second: the output order of the forward kernels)
constexpr int cart_index(int L, int c0, int c1) { return (L - c0) * (L - c0 + 1) / 2 + (L - c0 - c1); }

template <int A, int B, int Cc, int D>
constexpr BwdTab<A, B, Cc, D> make_bwd_tab() {
    using T = BwdTab<A, B, Cc, D>;
    T t{};
    constexpr int LC1 = T::LC1, LD1 = T::LD1, JLP = T::JLP;
    int n = 0;
    for (int w = 0; w < T::WN; ++w) {
        const int i3 = w % T::W4, i2 = (w / T::W4) % T::W3, i1 = (w / (T::W4 * T::W3)) % T::W2,
                  i0 = w / (T::W4 * T::W3 * T::W2);
        t.start[w] = (unsigned short)n;
        for (int ay = 0; ay <= A - i0; ++ay)
            for (int by = 0; by <= B - i1; ++by)
                for (int cy = 0; cy <= Cc - i2; ++cy)
                    for (int dy = 0; dy <= D - i3; ++dy) {
                        const int az = A - i0 - ay, bz = B - i1 - by, cz = Cc - i2 - cy, dz = D - i3 - dy;
                        const unsigned long long yo = (unsigned long long)((ay * LC1 + cy) * JLP + by * LD1 + dy);
                        const unsigned long long zo = (unsigned long long)((az * LC1 + cz) * JLP + bz * LD1 + dz);
                        for (int x = 0; x < 3; ++x) {
                            const int y = x == 2 ? 0 : x + 1;
                            const int a0 = x == 0 ? i0 : (y == 0 ? ay : az), a1 = x == 1 ? i0 : (y == 1 ? ay : az);
                            const int b0 = x == 0 ? i1 : (y == 0 ? by : bz), b1 = x == 1 ? i1 : (y == 1 ? by : bz);
                            const int c0 = x == 0 ? i2 : (y == 0 ? cy : cz), c1 = x == 1 ? i2 : (y == 1 ? cy : cz);
                            const int d0 = x == 0 ? i3 : (y == 0 ? dy : dz), d1 = x == 1 ? i3 : (y == 1 ? dy : dz);
                            const int g = ((cart_index(A, a0, a1) * T::NB + cart_index(B, b0, b1)) * T::NC +
                                           cart_index(Cc, c0, c1)) * T::ND + cart_index(D, d0, d1);
                            t.e[x * T::N + n] = (unsigned long long)g | (yo << 16) | (zo << 32);
                        }
                        ++n;
                    }
    }
    t.start[T::WN] = (unsigned short)n;
    return t;
}

}  // namespace eri
