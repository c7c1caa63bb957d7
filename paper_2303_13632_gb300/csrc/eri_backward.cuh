// eri_backward.cuh -- adjoint of the ERI kernel: gradients of E = sum_q sum_abcd G_abcd (ab|cd)
// with respect to the shell centres and the primitive exponents, recomputing the recurrences.
//
// For a primitive g_a = c N(alpha, L) prod_xi (r_xi - A_xi)^{a_xi} exp(-alpha |r - A|^2):
//   d g_a / d A_xi  = 2 alpha g_{a + 1_xi} - a_xi g_{a - 1_xi}
//   d g_a / d alpha = (2L + 3) / (4 alpha) g_a - sum_xi g_{a + 2_xi}
// (shifted functions keep the coefficient and normalisation of g_a).  In the Rys form of
// Eq. 8 each shift touches one axis factor only, so with the 2-D integrals I(i,j,k,l,mu,xi)
// built for every index up to L + 2 (VRR Eq. 6 and HRR Eq. 7 on the extended ranges, n_Rys =
// floor((L+2)/2) + 1 roots, exact for the shifted integrals of total degree <= L + 2):
//   dE/dA_x = sum_mu sum_abcd G_abcd [2 alpha Ix(a+1) - a_x Ix(a-1)] Iy Iz, likewise y, z, B, C, D
//   dE/d alpha_a = sum_mu sum_abcd G_abcd [(2La+3)/(4 alpha) Ix Iy Iz - Ix(a+2) Iy Iz - ...].
// Centre gradients are summed over primitives; exponent gradients go to the primitive.
#pragma once

#include "eri_bwd_table.h"
#include "eri_kernels.cuh"

namespace eri {

// 2-D integral configuration on the extended index ranges (all L + 2) of class (La..Ld), in
// the recurrence type R: FP64 keeps the VRR + HRR of Eqs. 6-7; FP32 (the mixed adjoint) uses the
// four-index recursion of phase_direct, which does not amplify FP32 rounding through the
// transfer relation (see eri_kernels.cuh), with the B and C values of the mixed setup.
template <int La0, int Lb0, int Lc0, int Ld0, typename R_ = double>
struct GCfg {
    using R = R_;
    static constexpr int oLa = La0, oLb = Lb0, oLc = Lc0, oLd = Ld0;
    static constexpr int oNA = ncart(La0), oNB = ncart(Lb0), oNC = ncart(Lc0), oND = ncart(Ld0);
    static constexpr int oNERI = oNA * oNB * oNC * oND;
    static constexpr int La = La0 + 2, Lb = Lb0 + 2, Lc = Lc0 + 2, Ld = Ld0 + 2;
    static constexpr int NAB = La + Lb, NCD = Lc + Ld;
    static constexpr int NRYS = (La0 + Lb0 + Lc0 + Ld0 + 2) / 2 + 1;
    static constexpr int RB = (int)sizeof(R);
    static constexpr bool FUSE_BC = false;
    static constexpr bool DIRECT = sizeof(R) == 4;
    static constexpr bool SWAB_OK = !DIRECT, SWCD_OK = !DIRECT;
    static constexpr int S_CB = S_N;
    static constexpr int S_CD = S_N + (DIRECT ? 3 : 0);
    static constexpr int SN = S_CD + (DIRECT ? 3 : 0);
    static constexpr int JL = (Lb + 1) * (Ld + 1);
    static constexpr int IBLK = (La + 1) * (Lc + 1) * JL;
    static constexpr int JLP = (JL % 2) ? JL : JL + 1;
    static constexpr int IBLKP = (La + 1) * (Lc + 1) * JLP;
    static constexpr int HBLK = (La + 1) * (Lb + 1) * (NCD + 1);
    static constexpr int GEO_BYTES = G_N * 8;
    static constexpr int BC_BYTES = NRYS * SN * RB;
    static constexpr int H_BYTES = DIRECT ? 0 : 3 * NRYS * HBLK * RB;
    static constexpr int I_BYTES = 3 * NRYS * IBLKP * RB;
    static constexpr int NACC = 17;  // dR[4][3], dalpha-part[4], E
    static constexpr int PERQ = GEO_BYTES + RG_N * RB + BC_BYTES + H_BYTES + I_BYTES + NACC * 8 +
                                oNERI * RB + 160;
    static constexpr int Q = imax(1, imin(8, (100 * 1024) / PERQ));
    static constexpr int THREADS = 256;
    static constexpr int OFF_GEO = 0;
    static constexpr int OFF_RG = Q * GEO_BYTES;
    static constexpr int OFF_BC = ((OFF_RG + Q * RG_N * RB + 15) / 16) * 16;
    static constexpr int OFF_ACC = ((OFF_BC + Q * BC_BYTES + 15) / 16) * 16;
    static constexpr int OFF_DR = OFF_ACC + Q * NACC * 8;        // centre gradients, all primitives
    static constexpr int OFF_PRIM = OFF_DR + Q * 12 * 8;          // primitive ids + exponents
    static constexpr int OFF_H = ((OFF_PRIM + Q * 8 * 8 + 15) / 16) * 16;
    static constexpr int OFF_I = OFF_H + Q * H_BYTES;
    static constexpr int OFF_G = OFF_I + Q * I_BYTES;  // the tile's upstream G, generic order
    static constexpr int SMEM = OFF_G + Q * oNERI * RB + 16;
};

template <class C>
__device__ __forceinline__ typename C::R gI(const typename C::R *Iq, int xi, int mu, int i, int j, int k,
                                            int l) {
    return Iq[i_index<C>(xi, mu, i, k, j, l)];
}

// The index table of the grouped contraction (eri_bwd_table.h), as device data, one per canonical
// class.
template <int A, int B, int Cc, int D>
__device__ const BwdTab<A, B, Cc, D> kBwdTab = make_bwd_tab<A, B, Cc, D>();

template <class C>
__device__ __forceinline__ void backward_tile(const ShellsDev &sh, const Tables &tb,
                                              const ClassArgs &args, const double *__restrict__ G,
                                              double *__restrict__ dR, double *__restrict__ dalpha) {
    using R = typename C::R;
    extern __shared__ __align__(16) unsigned char smem[];
    double *geo_s = reinterpret_cast<double *>(smem + C::OFF_GEO);
    R *rg_s = reinterpret_cast<R *>(smem + C::OFF_RG);
    R *bc_s = reinterpret_cast<R *>(smem + C::OFF_BC);
    double *acc_s = reinterpret_cast<double *>(smem + C::OFF_ACC);
    double *dr_s = reinterpret_cast<double *>(smem + C::OFF_DR);
    double *prim_s = reinterpret_cast<double *>(smem + C::OFF_PRIM);  // [q][0..3] exps, [4..7] prim ids
    R *H_s = reinterpret_cast<R *>(smem + C::OFF_H);
    R *I_s = reinterpret_cast<R *>(smem + C::OFF_I);
    __shared__ int maxprim_s;
    __shared__ int4 qt_s[C::Q];
    __shared__ R ea_s[C::Q * 4];  // 2 alpha of the quartet's four primitives, in R

    const int tid = threadIdx.x;
    const long long q0 = (long long)blockIdx.x * C::Q;
    const int qn = (int)((args.nq - q0) < C::Q ? (args.nq - q0) : C::Q);
    if (tid == 0) maxprim_s = 1;
    for (int i = tid; i < C::Q * 12; i += C::THREADS) dr_s[i] = 0.0;
    for (int q = tid; q < C::Q; q += C::THREADS) {
        int4 g = q < qn ? args.quartets[q0 + q] : make_int4(0, 0, 0, 0);
        qt_s[q] = make_int4(pick(g, args.perm[0]), pick(g, args.perm[1]), pick(g, args.perm[2]),
                            pick(g, args.perm[3]));
    }
    // the tile's G (contiguous per quartet in the class's generic layout), read once for all
    // primitives into the canonical component order (rounded to FP32 once for the mixed adjoint)
    R *G_s = reinterpret_cast<R *>(smem + C::OFF_G);
    {
        const int st0 = args.ostride[0], st1 = args.ostride[1], st2 = args.ostride[2],
                  st3 = args.ostride[3];
        for (int t = tid; t < qn * C::oNERI; t += C::THREADS) {
            const int q = t / C::oNERI, e = t - q * C::oNERI;
            const int id = e % C::oND, ic = (e / C::oND) % C::oNC, ib = (e / (C::oND * C::oNC)) % C::oNB,
                      ia = e / (C::oND * C::oNC * C::oNB);
            G_s[t] = to_r<R>(G[(q0 + q) * C::oNERI + ia * st0 + ib * st1 + ic * st2 + id * st3]);
        }
    }
    __syncthreads();

    for (int prim = 0; prim < maxprim_s; ++prim) {
        for (int i = tid; i < C::Q * C::NACC; i += C::THREADS) acc_s[i] = 0.0;
        for (int q = tid; q < C::Q; q += C::THREADS) {
            double *geo = geo_s + q * G_N;
            int np = 0;
            if (q < qn) {
                int4 qt = qt_s[q];
                phase_geometry<C>(sh, qt, prim, geo, np);
                if (prim < np) {
                    int nb = sh.nprim[qt.y], nc = sh.nprim[qt.z], nd = sh.nprim[qt.w];
                    int id = prim % nd, t = prim / nd;
                    int ic = t % nc;
                    t /= nc;
                    int ib = t % nb, ia = t / nb;
                    int pk[4] = {sh.pofs[qt.x] + ia, sh.pofs[qt.y] + ib, sh.pofs[qt.z] + ic,
                                 sh.pofs[qt.w] + id};
                    for (int k = 0; k < 4; ++k) {
                        prim_s[q * 8 + k] = sh.exps[pk[k]];
                        prim_s[q * 8 + 4 + k] = (double)pk[k];
                        ea_s[q * 4 + k] = to_r<R>(2.0 * sh.exps[pk[k]]);
                    }
                }
            } else {
                geo[G_PREF] = 0.0;
                geo[G_T] = 0.0;
                for (int s = G_P; s < G_N; ++s)
                    geo[s] = (s == G_P || s == G_Q || s == G_IP || s == G_IQ) ? 1.0
                                                                              : (s == G_IPQ ? 0.5 : 0.0);
            }
            if (prim == 0 && np > 1) atomicMax(&maxprim_s, np);
            R *rg = rg_s + q * RG_N;
            rg[RG_ABX] = to_r<R>(geo[G_ABX]);
            rg[RG_ABY] = to_r<R>(geo[G_ABY]);
            rg[RG_ABZ] = to_r<R>(geo[G_ABZ]);
            rg[RG_CDX] = to_r<R>(geo[G_CDX]);
            rg[RG_CDY] = to_r<R>(geo[G_CDY]);
            rg[RG_CDZ] = to_r<R>(geo[G_CDZ]);
            rg[RG_SWAB] = to_r<R>(geo[G_SWAB]);
            rg[RG_SWCD] = to_r<R>(geo[G_SWCD]);
            if (q >= qn || prim >= np) {
                for (int k = 0; k < 4; ++k) {
                    prim_s[q * 8 + k] = 1.0;
                    prim_s[q * 8 + 4 + k] = -1.0;
                    ea_s[q * 4 + k] = (R)2;
                }
            }
        }
        __syncthreads();
        for (int it = tid; it < C::Q * C::NRYS; it += C::THREADS) {
            int q = it / C::NRYS, mu = it % C::NRYS;
            phase_setup<C>(tb, geo_s + q * G_N, mu, bc_s + (q * C::NRYS + mu) * C::SN);
        }
        __syncthreads();
        for (int it = tid; it < C::Q * C::NRYS * 3; it += C::THREADS) {
            int q = it / (C::NRYS * 3), r = it % (C::NRYS * 3);
            if constexpr (C::DIRECT)
                phase_direct<C>(bc_s + q * C::NRYS * C::SN, r / 3, r % 3, I_s + (size_t)q * (C::I_BYTES / C::RB));
            else
                phase_vrr<C>(bc_s + q * C::NRYS * C::SN, rg_s + q * RG_N, r / 3, r % 3,
                             H_s + (size_t)q * (C::H_BYTES / C::RB), I_s + (size_t)q * (C::I_BYTES / C::RB));
        }
        __syncthreads();
        if constexpr (!C::DIRECT) {
            constexpr int NIJ = (C::La + 1) * (C::Lb + 1);
            for (int it = tid; it < C::Q * C::NRYS * 3 * NIJ; it += C::THREADS) {
                int q = it / (C::NRYS * 3 * NIJ), r = it % (C::NRYS * 3 * NIJ);
                int mu = r / (3 * NIJ);
                r %= 3 * NIJ;
                int xi = r / NIJ, ij = r % NIJ;
                phase_ket<C>(rg_s + q * RG_N, mu, xi, ij / (C::Lb + 1), ij % (C::Lb + 1),
                             H_s + (size_t)q * (C::H_BYTES / C::RB), I_s + (size_t)q * (C::I_BYTES / C::RB));
            }
            __syncthreads();
        }
        // contraction with G, grouped by axis: for axis x and the x-components (i0, i1, i2, i3)
        // of the four centres, W = sum of G I_y I_z over the outputs with those x-components
        // (y, z the other two axes); each derivative factor of axis x then multiplies W once
        // instead of once per output.
        {
            constexpr int W1 = C::oLa + 1, W2 = C::oLb + 1, W3 = C::oLc + 1, W4 = C::oLd + 1;
            constexpr int WN = W1 * W2 * W3 * W4;
            constexpr int ITEMS = C::NRYS * 3 * WN;
            const auto &tab = kBwdTab<C::oLa, C::oLb, C::oLc, C::oLd>;
            using Tab = BwdTab<C::oLa, C::oLb, C::oLc, C::oLd>;
            static_assert(Tab::WN == WN && Tab::N == C::oNERI && Tab::LC1 == C::Lc + 1 && Tab::LD1 == C::Ld + 1 &&
                              Tab::JLP == C::JLP,
                          "index table and 2-D integral layout disagree");
            const int lane = tid & 31;
            for (int q = 0; q < qn; ++q) {
                const R *Iq = I_s + (size_t)q * (C::I_BYTES / C::RB);
                const R *Gq = G_s + q * C::oNERI;
                R ea[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) ea[k] = ea_s[q * 4 + k];
                // the thread's sums (in R)
                R r[C::NACC];
#pragma unroll
                for (int k = 0; k < C::NACC; ++k) r[k] = (R)0;
                for (int it = tid; it < ITEMS; it += C::THREADS) {
                    const int mu = it / (3 * WN), rem = it % (3 * WN);
                    const int x = rem / WN, w = rem % WN;
                    const int i3 = w % W4, i2 = (w / W4) % W3, i1 = (w / (W4 * W3)) % W2,
                              i0 = w / (W4 * W3 * W2);
                    const int y = x == 2 ? 0 : x + 1, z = x == 0 ? 2 : x - 1;
                    const R *Iy = Iq + i_index<C>(y, mu, 0, 0, 0, 0), *Iz = Iq + i_index<C>(z, mu, 0, 0, 0, 0);
                    const unsigned long long *ent = tab.e + x * C::oNERI;
                    R W = (R)0;
                    for (int k = tab.start[w], k1 = tab.start[w + 1]; k < k1; ++k) {
                        const unsigned long long v = ent[k];
                        W = fma(Gq[(int)(v & 0xffffu)] * Iy[(int)((v >> 16) & 0xffffu)], Iz[(int)(v >> 32)], W);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int nk = k == 0 ? i0 : (k == 1 ? i1 : (k == 2 ? i2 : i3));
                        const int e0 = (k == 0), e1 = (k == 1), e2 = (k == 2), e3 = (k == 3);
                        const R up = gI<C>(Iq, x, mu, i0 + e0, i1 + e1, i2 + e2, i3 + e3);
                        const R up2 = gI<C>(Iq, x, mu, i0 + 2 * e0, i1 + 2 * e1, i2 + 2 * e2, i3 + 2 * e3);
                        const R dn = nk > 0 ? gI<C>(Iq, x, mu, i0 - e0, i1 - e1, i2 - e2, i3 - e3) : (R)0;
                        const R t = W * (ea[k] * up - (R)nk * dn);
                        // r[k * 3 + x] with x known only at run time: select, no dynamic indexing
                        r[k * 3 + 0] += x == 0 ? t : (R)0;
                        r[k * 3 + 1] += x == 1 ? t : (R)0;
                        r[k * 3 + 2] += x == 2 ? t : (R)0;
                        r[12 + k] -= W * up2;
                    }
                    if (x == 0) r[16] += W * gI<C>(Iq, 0, mu, i0, i1, i2, i3);
                }
                // warp sums in R (FP32 in the mixed adjoint: the FP64 pipe is the scarce one there),
                // then FP64 across warps, primitives and quartets
#pragma unroll
                for (int k = 0; k < C::NACC; ++k) {
                    R v = r[k];
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
                    if (lane == 0 && v != (R)0) atomicAdd(acc_s + q * C::NACC + k, RTraits<R>::to_f64(v));
                }
            }
        }
        __syncthreads();
        // per quartet: exponent gradients of this primitive quartet, centre gradients summed
        for (int q = tid; q < qn; q += C::THREADS) {
            const double *acc = acc_s + q * C::NACC;
            const double *ex = prim_s + q * 8;
            const int Lk[4] = {C::oLa, C::oLb, C::oLc, C::oLd};
            if (ex[4] >= 0.0) {
                for (int k = 0; k < 4; ++k) {
                    double v = (2.0 * Lk[k] + 3.0) / (4.0 * ex[k]) * acc[16] + acc[12 + k];
                    atomicAdd(dalpha + (long long)ex[4 + k], v);
                }
                for (int i = 0; i < 12; ++i) dr_s[q * 12 + i] += acc[i];
            }
        }
        __syncthreads();
    }
    for (int it = tid; it < qn * 12; it += C::THREADS) {
        int q = it / 12, i = it % 12, k = i / 3, x = i % 3;
        int4 qt = qt_s[q];
        int s = pick(qt, k);
        atomicAdd(dR + 3LL * s + x, dr_s[q * 12 + i]);
    }
}

template <class C>
__global__ void __launch_bounds__(C::THREADS)
eri_backward_kernel(ShellsDev sh, Tables tb, ClassArgs args, const double *__restrict__ G,
                    double *__restrict__ dR, double *__restrict__ dalpha) {
    backward_tile<C>(sh, tb, args, G, dR, dalpha);
}

// The same for the mixed adjoint of classes with an f shell, compiled for one resident CTA per
// SM: under the default bound ptxas caps some of them at 128 registers with large spills, and
// [ff|pp] then returned wrong exponent gradients for its first centre (the emulated kernel
// arithmetic and the oracle agree); with the whole register file available none spills.
template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
eri_backward_kernel_wide(ShellsDev sh, Tables tb, ClassArgs args, const double *__restrict__ G,
                         double *__restrict__ dR, double *__restrict__ dalpha) {
    backward_tile<C>(sh, tb, args, G, dR, dalpha);
}

template <int La, int Lb, int Lc, int Ld, typename R = double>
cudaError_t launch_backward(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                            const double *G, double *dR, double *dalpha, cudaStream_t stream) {
    using C = GCfg<La, Lb, Lc, Ld, R>;
    static_assert(C::SMEM <= 227 * 1024, "adjoint tile exceeds shared memory");
    if (args.nq <= 0) return cudaSuccess;
    constexpr bool wide = sizeof(R) == 4 && (La == 3 || Lb == 3 || Lc == 3 || Ld == 3);
    void (*kern)(ShellsDev, Tables, ClassArgs, const double *, double *, double *);
    if constexpr (wide)
        kern = eri_backward_kernel_wide<C>;
    else
        kern = eri_backward_kernel<C>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    long long grid = (args.nq + C::Q - 1) / C::Q;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, C::THREADS, C::SMEM, stream>>>(sh, tb, args, G, dR, dalpha);
    return cudaGetLastError();
}

}  // namespace eri
