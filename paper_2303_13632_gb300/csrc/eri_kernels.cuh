// eri_kernels.cuh -- class-templated ERI kernel: Rys quadrature fused with compression.
//
// arXiv 2303.13632, Sec. III-B: one kernel per quartet class (La, Lb, Lc, Ld), the
// angular momenta being compile-time parameters from which n_g and n_Rys follow.
// Per primitive quartet the kernel runs the stages of Sec. II-C / Fig. 1:
//   setup      B00, B10, B01 and C00_xi, C00'_xi for each root (the B and C arrays),
//   VRR        Eq. 6: I(i+1,0,k,0) = i B10 I(i-1,..) + k B00 I(i,..,k-1) + C00 I(i,..,k)
//                     I(i,0,k+1,0) = k B01 I(..,k-1) + i B00 I(i-1,..,k) + C00' I(i,..,k)
//   HRR        Eq. 7: I(i,j,k,l) = I(i+1,j-1,k,l) + (A-B)_xi I(i,j-1,k,l), then the same on
//                     the ket with (C-D)_xi,
//   quadrature Eq. 8: [ab|cd] = sum_mu prod_xi I(a_xi, b_xi, c_xi, d_xi, mu, xi), with the
//                     weight and the Gaussian-product prefactor folded into the z origin,
// sums the primitive quartets (contraction), and then either stores FP64 values or
// compresses each quartet (Sec. II-D): b_max (max |x|), eps = b_max / (2^{n-1}-1) (Eq. 9),
// q = ANINT(x eps^{-1}) (Eq. 10), packed into an n-bit little-endian stream.
//
// GPU mapping (replaces the FPGA's pipelined loops and private buffer copies, Sec. III-C..E):
// a CTA owns a tile of Q quartets of one class and runs the stages as data-parallel phases
// separated by __syncthreads():
//   A0 geometry + prefactor   one thread per quartet                      (FP64)
//   A1 roots/weights + B, C   one thread per (quartet, root)              (FP64 -> R)
//   B  VRR + bra HRR          one thread per (quartet, root, axis)        (R)
//   C  ket HRR                one thread per (quartet, root, axis, i, j)  (R)
//   D  quadrature             one thread per (quartet, a, c, b-chunk), the b-chunk x d
//                             outputs held in registers across primitives (R)
//   E  b_max, eps, quantise, pack through shared memory, store          (compressed mode)
// The intermediates I(i,j,k,l,mu,xi) of Table I live in shared memory; several CTAs per SM
// overlap their phases, which is the GPU analogue of the paper's c_max concurrent quartets.
// R = double gives the plain FP64 path, R = float the mixed path (FP64 setup/roots, FP32
// recurrences and quadrature, Kahan-compensated sums over primitives).
#pragma once

#include "eri_device.cuh"

namespace eri {

template <typename R>
struct RTraits;
template <>
struct RTraits<double> {
    static __device__ __forceinline__ double round_away(double v) { return round(v); }
    static __device__ __forceinline__ double to_f64(double v) { return v; }
    static __device__ __forceinline__ bool finite(double v) { return fabs(v) <= 1.7976931348623157e308; }
};
template <>
struct RTraits<float> {
    static __device__ __forceinline__ float round_away(float v) { return roundf(v); }
    static __device__ __forceinline__ double to_f64(float v) { return f32_to_f64(v); }
    static __device__ __forceinline__ bool finite(float v) { return fabsf(v) <= 3.4028234663852886e38f; }
};

// Two's complement bits of an integral value |v| <= 2^{bits-1} - 1.  In FP32 and for widths up
// to 23 the sum v + 1.5 * 2^23 is exact and its low mantissa bits are the integer, which
// replaces a float-to-integer conversion instruction per value by one FP32 add.
template <typename R>
__device__ __forceinline__ uint32_t to_code(R v, int bits) {
    if constexpr (sizeof(R) == 4) {
        if (bits <= 23) return (uint32_t)(__float_as_int(v + 12582912.0f) - 0x4B400000);
    }
    return (uint32_t)(int)v;
}

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr int imin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }
// smallest b-chunk >= b with nanc * ceil(nb / chunk) <= 1024 phase-D items per quartet
__host__ __device__ constexpr int bch_fit(int nanc, int nb, int b) {
    while (b < nb && nanc * cdiv(nb, b) > 1024) ++b;
    return b;
}

// ids[k] of an int4 without dynamic register indexing.
__device__ __forceinline__ int pick(const int4 &g, int k) {
    return k == 0 ? g.x : (k == 1 ? g.y : (k == 2 ? g.z : g.w));
}

// Per-quartet geometry kept in shared memory (FP64).
// G_SWAB / G_SWCD = 1 when the VRR is built on B (D) and the HRR transfers to a (c); see
// phase_geometry.
enum GeoSlot {
    G_T = 0, G_PREF, G_P, G_Q, G_PAX, G_PAY, G_PAZ, G_QCX, G_QCY, G_QCZ, G_PQX, G_PQY, G_PQZ,
    G_ABX, G_ABY, G_ABZ, G_CDX, G_CDY, G_CDZ, G_SWAB, G_SWCD, G_IP, G_IQ, G_IPQ, G_N
};
// Per-quartet geometry the recurrence stages read, in the recurrence type R (no FP64 there).
enum RGeoSlot { RG_ABX = 0, RG_ABY, RG_ABZ, RG_CDX, RG_CDY, RG_CDZ, RG_SWAB, RG_SWCD, RG_N };
// Per (quartet, root) setup values kept in shared memory (type R).  S_C0 / S_C1 are C00 and
// C00' relative to the centres the recurrence is built on; classes on the four-index path
// (Cfg::DIRECT) append C00 relative to B (at Cfg::S_CB, when Lb > 0) and C00' relative to D
// (at Cfg::S_CD, when Ld > 0), Cfg::SN values in all.
enum BCSlot { S_B00 = 0, S_B10, S_B01, S_C0X, S_C0Y, S_C0Z, S_C1X, S_C1Y, S_C1Z, S_WZ, S_N };

template <int La_, int Lb_, int Lc_, int Ld_, typename R_>
struct Cfg {
    using R = R_;
    static constexpr int La = La_, Lb = Lb_, Lc = Lc_, Ld = Ld_;
    static constexpr int NA = ncart(La), NB = ncart(Lb), NC = ncart(Lc), ND = ncart(Ld);
    static constexpr int NERI = NA * NB * NC * ND;
    static constexpr int NRYS = (La + Lb + Lc + Ld) / 2 + 1;
    static constexpr int NAB = La + Lb, NCD = Lc + Ld;
    static constexpr int JL = (Lb + 1) * (Ld + 1);          // I block for fixed (xi, mu, i, k)
    static constexpr int IBLK = (La + 1) * (Lc + 1) * JL;   // I per (xi, mu)
    // shared-memory strides: blocks padded to an odd number of elements so that the blocks
    // the lanes of a warp read in phase D start in different banks
    static constexpr int JLP = (JL % 2) ? JL : JL + 1;
    static constexpr int IBLKP = (La + 1) * (Lc + 1) * JLP;
    static constexpr int HBLK = (La + 1) * (Lb + 1) * (NCD + 1);  // bra-transferred per (xi, mu)
    static constexpr bool FUSE_BC = HBLK <= 48;             // ket HRR in registers in phase B
    // thread-per-quartet kernels (all intermediates in registers): with the FP64 setup inline
    // for the small classes (TPQ_SMALL); in FP32 up to 100 outputs, reading the records of the
    // split path's setup kernel (TPQ_SPLIT)
    static constexpr bool TPQ_SMALL = (sizeof(R) == 4 ? NERI <= 36 : NERI <= 18) && IBLK <= 16;
    static constexpr bool TPQ_SPLIT = sizeof(R) == 4 && !TPQ_SMALL && NERI <= 100 && IBLK <= 16;
    static constexpr bool TPQ = TPQ_SMALL || TPQ_SPLIT;
    // primitive (K = 1) plans run the class through the setup kernel
    static constexpr bool USES_SETUP = !TPQ_SMALL;
    // FP32 recurrences with angular momentum on b or d use the four-index recursion
    // (phase_direct, axis_direct): in FP32 the transfer relation amplifies rounding by up to
    // about 3^(Lb+Ld).  FP64 and the small inline-setup classes keep the VRR + HRR of Eqs. 6-7.
    static constexpr bool DIRECT = sizeof(R) == 4 && !TPQ_SMALL && (Lb + Ld) > 0;
    // VRR built on B (D) with the HRR transferring to a (c) where that is the better-
    // conditioned direction; never when b (d) carries no angular momentum
    static constexpr bool SWAB_OK = !DIRECT && Lb > 0;
    static constexpr bool SWCD_OK = !DIRECT && Ld > 0;
    static constexpr int S_CB = S_N;
    static constexpr int S_CD = S_N + (DIRECT && Lb > 0 ? 3 : 0);
    static constexpr int SN = S_CD + (DIRECT && Ld > 0 ? 3 : 0);
    static constexpr int RWORDS = sizeof(R) / 4;
    // outputs per thread: bchunk x ND accumulators (+ Kahan compensation in FP32)
    static constexpr int ACC_REGS = (sizeof(R) == 8) ? 48 : 64;
    // widened where one thread per phase-D item would exceed a CTA's 1024 threads (FP64 classes
    // with two g shells)
    static constexpr int BCH = bch_fit(NA * NC, NB, imax(1, imin(NB, ACC_REGS / (ND * RWORDS))));
    static constexpr int NCH = cdiv(NB, BCH);
    static constexpr int ITEMS_D = NA * NC * NCH;
    // shared memory per quartet (bytes)
    static constexpr int GEO_BYTES = G_N * 8;
    static constexpr int BC_BYTES = NRYS * SN * (int)sizeof(R);
    static constexpr int H_BYTES = (FUSE_BC || DIRECT) ? 0 : 3 * NRYS * HBLK * (int)sizeof(R);
    static constexpr int I_BYTES = 3 * NRYS * IBLKP * (int)sizeof(R);
    static constexpr int STAGE_BYTES = NERI * 3;  // worst case 24-bit codes
    static constexpr int UNION_BYTES = imax(H_BYTES + I_BYTES, STAGE_BYTES);
    static constexpr int PERQ = GEO_BYTES + RG_N * (int)sizeof(R) + BC_BYTES + UNION_BYTES + 8;
    static constexpr int SMEM_BUDGET = 96 * 1024;
    static constexpr int QMAX_T = imax(1, 256 / ITEMS_D);
    static constexpr int QMAX_S = imax(1, SMEM_BUDGET / PERQ);
    static constexpr int Q = imin(128, imin(QMAX_T, QMAX_S));
    static constexpr int THREADS = imax(64, cdiv(Q * ITEMS_D, 32) * 32);
    // shared memory layout (byte offsets)
    static constexpr int OFF_GEO = 0;
    static constexpr int OFF_RG = OFF_GEO + Q * GEO_BYTES;
    static constexpr int OFF_BC = ((OFF_RG + Q * RG_N * (int)sizeof(R) + 15) / 16) * 16;
    static constexpr int OFF_BMAX = ((OFF_BC + Q * BC_BYTES + 15) / 16) * 16;
    static constexpr int OFF_U = ((OFF_BMAX + Q * 8 + 15) / 16) * 16;
    static constexpr int OFF_H = OFF_U;
    static constexpr int OFF_I = OFF_U + Q * H_BYTES;
    static constexpr int SMEM = OFF_U + ((Q * UNION_BYTES + 16 + 15) / 16) * 16 + 16;
    // values per quartet written by the separate setup kernel (K = 1 plans)
    static constexpr int SETUP_GEO = 8;  // AB, CD, swab, swcd
    static constexpr int SETUP_FIELDS = SETUP_GEO + NRYS * SN;
    static constexpr int TPQ_THREADS = 128;
    // resident CTAs per SM the thread-per-quartet kernel is compiled for (the register cap):
    // the inline-setup FP32 kernels wait on two random pair-table records per quartet, so they
    // need more warps in flight than their natural register use (about 100) allows.  The caps
    // are the largest at which ptxas reports no spill for these classes (8 CTAs = 64 registers
    // up to 6 outputs, 7 = 72 up to 10, 6 = 80 up to 18; larger classes keep their own count).
    // [ss|ss] measured 6% slower at 8 CTAs than with its own count and keeps it.
    // the inline-setup FP32 kernels form B and C per root in two-float FP32 (SetupTF) from two
    // roots on; with one root the FP64 evaluation is cheaper than the per-quartet splitting.
    // [ds|ds] and [dp|ss] measured 14% and 3% slower with it (more registers, fewer resident
    // CTAs) and keep the FP64 evaluation.
    static constexpr bool TF_SLOWER = (La == 2 && Lb == 0 && Lc == 2 && Ld == 0) ||
                                      (La == 2 && Lb == 1 && Lc == 0 && Ld == 0);
    static constexpr bool SETUP_TF = sizeof(R) == 4 && NRYS >= 2 && !TF_SLOWER;
    static constexpr int TPQ_MINB = (TPQ_SMALL && sizeof(R) == 4)
                                        ? (NERI == 1 ? 1 : (NERI <= 6 ? 8 : (NERI <= 10 ? 7 : (NERI <= 18 ? 6 : 1))))
                                        : 1;
};

// ---------------------------------------------------------------------------------------
// Phase A0: geometry and prefactor of primitive quartet `prim` of quartet q.
template <class C>
__device__ __forceinline__ void phase_geometry(const ShellsDev &sh, const int4 &qt, int prim,
                                               double *geo, int &nprim_total) {
    int na = sh.nprim[qt.x], nb = sh.nprim[qt.y], nc = sh.nprim[qt.z], nd = sh.nprim[qt.w];
    nprim_total = na * nb * nc * nd;
    if (prim >= nprim_total) {
        geo[G_PREF] = 0.0;
        geo[G_T] = 0.0;
        for (int s = G_P; s < G_N; ++s)
            geo[s] = (s == G_P || s == G_Q || s == G_IP || s == G_IQ) ? 1.0 : (s == G_IPQ ? 0.5 : 0.0);
        return;
    }
    int id = prim % nd, t = prim / nd;
    int ic = t % nc;
    t /= nc;
    int ib = t % nb, ia = t / nb;
    int pa = sh.pofs[qt.x] + ia, pb = sh.pofs[qt.y] + ib, pc = sh.pofs[qt.z] + ic,
        pd = sh.pofs[qt.w] + id;
    double ea = sh.exps[pa], eb = sh.exps[pb], ec = sh.exps[pc], ed = sh.exps[pd];
    double A[3] = {sh.cx[qt.x], sh.cy[qt.x], sh.cz[qt.x]};
    double B[3] = {sh.cx[qt.y], sh.cy[qt.y], sh.cz[qt.y]};
    double Cc[3] = {sh.cx[qt.z], sh.cy[qt.z], sh.cz[qt.z]};
    double D[3] = {sh.cx[qt.w], sh.cy[qt.w], sh.cz[qt.w]};
    double p = ea + eb, q = ec + ed;
    // 1/p and 1/q from one FP64 division; 1/(p+q) as rsqrt(p+q)^2 (no second division)
    const double pq = p * q;
    const double ipq_prod = 1.0 / pq;
    const double ip = q * ipq_prod, iq = p * ipq_prod;
    const double rs = rsqrt(p + q);
    double ab2 = 0.0, cd2 = 0.0, pq2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double AB = A[x] - B[x], CD = Cc[x] - D[x];
        // P - A = -eb/p (A - B), Q - C = -ed/q (C - D): computed from differences
        double PA = -eb * ip * AB, QC = -ed * iq * CD;
        double PQ = (A[x] + PA) - (Cc[x] + QC);
        // the VRR is built on the centre nearer to P (the larger exponent): P - B = (P - A) + AB
        geo[G_PAX + x] = (C::SWAB_OK && eb > ea) ? PA + AB : PA;
        geo[G_QCX + x] = (C::SWCD_OK && ed > ec) ? QC + CD : QC;
        geo[G_PQX + x] = PQ;
        geo[G_ABX + x] = AB;
        geo[G_CDX + x] = CD;
        ab2 += AB * AB;
        cd2 += CD * CD;
        pq2 += PQ * PQ;
    }
    const double ipq = rs * rs;
    const double rho = pq * ipq;
    // K_AB K_CD = exp(-(ab/p |A-B|^2 + cd/q |C-D|^2)) in one FP64 exponential
    const double kabcd = exp(-(ea * eb * ip * ab2 + ec * ed * iq * cd2));
    // 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD times the four coef * N factors
    const double two_pi_52 = 34.986836655249725;
    geo[G_PREF] = two_pi_52 * ipq_prod * rs * kabcd * (sh.cn[pa] * sh.cn[pb]) *
                  (sh.cn[pc] * sh.cn[pd]);
    geo[G_T] = rho * pq2;
    geo[G_P] = p;
    geo[G_Q] = q;
    geo[G_SWAB] = (C::SWAB_OK && eb > ea) ? 1.0 : 0.0;
    geo[G_SWCD] = (C::SWCD_OK && ed > ec) ? 1.0 : 0.0;
    geo[G_IP] = ip;
    geo[G_IQ] = iq;
    geo[G_IPQ] = ipq;
}

// Phase A0 from the plan's primitive-pair table: the same geo values as phase_geometry, with
// the per-pair part (1/p, P - A, the exponential prefactor) read from the two pair records
// instead of recomputed for every quartet.
template <class C>
__device__ __forceinline__ void phase_geometry_pairs(const ShellsDev &sh,
                                                     const double *__restrict__ pairs,
                                                     long long np, const int4 &qt, int prim,
                                                     double *geo, int &nprim_total) {
    int na = sh.nprim[qt.x], nb = sh.nprim[qt.y], nc = sh.nprim[qt.z], nd = sh.nprim[qt.w];
    nprim_total = na * nb * nc * nd;
    if (prim >= nprim_total) {
        geo[G_PREF] = 0.0;
        geo[G_T] = 0.0;
        for (int s = G_P; s < G_N; ++s)
            geo[s] = (s == G_P || s == G_Q || s == G_IP || s == G_IQ) ? 1.0 : (s == G_IPQ ? 0.5 : 0.0);
        return;
    }
    int id = prim % nd, t = prim / nd;
    int ic = t % nc;
    t /= nc;
    int ib = t % nb, ia = t / nb;
    // 32-bit index arithmetic (64-bit integer operations issue on the FP64 pipe): the table
    // holds at most 16 GiB / 48 B < 2^32 / kPairFields records
    const unsigned int pa = sh.pofs[qt.x] + ia, pb = sh.pofs[qt.y] + ib, pc = sh.pofs[qt.z] + ic,
                       pd = sh.pofs[qt.w] + id, npu = (unsigned int)np;
    const double *rab = pairs + (pa * npu + pb) * (unsigned int)kPairFields;
    const double *rcd = pairs + (pc * npu + pd) * (unsigned int)kPairFields;
    const double p = __ldg(rab + PR_P), ip = __ldg(rab + PR_IP);
    const double q = __ldg(rcd + PR_P), iq = __ldg(rcd + PR_IP);
    bool swab = false, swcd = false;
    if constexpr (C::SWAB_OK) swab = __ldg(sh.exps + pb) > __ldg(sh.exps + pa);
    if constexpr (C::SWCD_OK) swcd = __ldg(sh.exps + pd) > __ldg(sh.exps + pc);
    double A[3] = {sh.cx[qt.x], sh.cy[qt.x], sh.cz[qt.x]};
    double B[3] = {sh.cx[qt.y], sh.cy[qt.y], sh.cz[qt.y]};
    double Cc[3] = {sh.cx[qt.z], sh.cy[qt.z], sh.cz[qt.z]};
    double D[3] = {sh.cx[qt.w], sh.cy[qt.w], sh.cz[qt.w]};
    const double rs = rsqrt(p + q);
    double pq2 = 0.0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        double AB = A[x] - B[x], CD = Cc[x] - D[x];
        double PA = __ldg(rab + PR_PAX + x), QC = __ldg(rcd + PR_PAX + x);
        double PQ = (A[x] + PA) - (Cc[x] + QC);
        geo[G_PAX + x] = swab ? PA + AB : PA;
        geo[G_QCX + x] = swcd ? QC + CD : QC;
        geo[G_PQX + x] = PQ;
        geo[G_ABX + x] = AB;
        geo[G_CDX + x] = CD;
        pq2 += PQ * PQ;
    }
    const double ipq = rs * rs;
    const double two_pi_52 = 34.986836655249725;
    geo[G_PREF] = two_pi_52 * (ip * iq) * rs * (__ldg(rab + PR_KCN) * __ldg(rcd + PR_KCN));
    geo[G_T] = (p * q * ipq) * pq2;
    geo[G_P] = p;
    geo[G_Q] = q;
    geo[G_SWAB] = swab ? 1.0 : 0.0;
    geo[G_SWCD] = swcd ? 1.0 : 0.0;
    geo[G_IP] = ip;
    geo[G_IQ] = iq;
    geo[G_IPQ] = ipq;
}

// Phase A0 dispatch: the pair table when the plan has one, else the full computation.
template <class C>
__device__ __forceinline__ void geometry_of(const ShellsDev &sh, const ClassArgs &args,
                                            const int4 &qt, int prim, double *geo,
                                            int &nprim_total) {
    if (args.pairs != nullptr)
        phase_geometry_pairs<C>(sh, args.pairs, args.np, qt, prim, geo, nprim_total);
    else
        phase_geometry<C>(sh, qt, prim, geo, nprim_total);
}

// Phase A1: root mu of quartet geometry geo -> B and C values (Rys setup stage), formed in
// FP64 and rounded to the recurrence type R.  C00 and C00' use the offsets of P and Q from the
// centres the VRR is built on (phase_geometry).  Classes with L = 0 need only F_0 (no root).
template <class C>
__device__ __forceinline__ void phase_setup(const Tables &tb, const double *geo, int mu,
                                            typename C::R *bc) {
    using R = typename C::R;
    constexpr int LTOT = C::NAB + C::NCD;
    double x, w;
    if constexpr (LTOT == 0) {
        double F0, F1;
        if constexpr (sizeof(R) == 4)
            boys_f01_mixed<false>(geo[G_T], tb.boys_t01, tb.boys_t01_f, F0, F1);
        else
            boys_f01<false>(geo[G_T], tb.boys_t01, F0, F1);
        w = F0;
        x = 0.0;
    } else {
        // mixed precision: the values are rounded to FP32 below, so the root evaluation of the
        // mixed setup (about 1e-9 relative) serves
        rys_root<sizeof(R) == 4>(tb, C::NRYS, mu, geo[G_T], x, w);
    }
    bc[S_WZ] = to_r<R>(geo[G_PREF] * w);
    if constexpr (LTOT > 0) {
        double p = geo[G_P], q = geo[G_Q];
        double ipq = geo[G_IPQ];
        double fq = q * x * ipq, fp = p * x * ipq;
        bc[S_B00] = to_r<R>(0.5 * x * ipq);
        bc[S_B10] = to_r<R>((1.0 - fq) * (0.5 * geo[G_IP]));
        bc[S_B01] = to_r<R>((1.0 - fp) * (0.5 * geo[G_IQ]));
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double pq = geo[G_PQX + s];
            bc[S_C0X + s] = to_r<R>(geo[G_PAX + s] - fq * pq);
            bc[S_C1X + s] = to_r<R>(geo[G_QCX + s] + fp * pq);
        }
        // four-index path: P - B = (P - A) + (A - B), Q - D = (Q - C) + (C - D)
        if constexpr (C::DIRECT && C::Lb > 0) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
                bc[C::S_CB + s] = to_r<R>((geo[G_PAX + s] + geo[G_ABX + s]) - fq * geo[G_PQX + s]);
        }
        if constexpr (C::DIRECT && C::Ld > 0) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
                bc[C::S_CD + s] = to_r<R>((geo[G_QCX + s] + geo[G_CDX + s]) + fp * geo[G_PQX + s]);
        }
    }
}

// Phase A1 of the mixed path for the roots of one (primitive) quartet computed by one thread:
// the root-independent factors of the B and C values are formed once per quartet and split
// into two-float form, so that each root costs FP32 work only:
//   B00 = x / (2(p+q)),  B10 = 1/(2p) - a10 x,  B01 = 1/(2q) - a01 x,
//   C00 = (P - A) - u x,  C00' = (Q - C) + v x,
//   a10 = q / (2p(p+q)),  a01 = p / (2q(p+q)),  u = q (P - Q) / (p+q),  v = p (P - Q) / (p+q).
// The differences that cancel are evaluated in two-float arithmetic, so the values keep the
// accuracy of the FP64 evaluation (rounded once to FP32) up to 2^-23 of the value plus 2^-46
// of the terms; the root x enters in two-float form as well.
template <class C>
struct SetupTF {
    static constexpr bool BRA = C::NAB > 0, KET = C::NCD > 0;
    static constexpr bool CB = C::DIRECT && C::Lb > 0, CD = C::DIRECT && C::Ld > 0;
    float hq, pref;
    F2 hip, a10, hiq, a01;
    F2 pa[3], u[3], qc[3], nv[3], pb[3], qd[3];

    __device__ __forceinline__ void init(const double *geo) {
        pref = f64_to_f32(geo[G_PREF]);
        if constexpr (BRA || KET) hq = 0.5f * f64_to_f32(geo[G_IPQ]);
        const double ipq = geo[G_IPQ];
        if constexpr (BRA) {
            const F2 ip = split_f2(geo[G_IP]), fq = split_f2(geo[G_Q] * ipq);
            hip = {0.5f * ip.h, 0.5f * ip.l};
            a10 = tf_mul(hip, fq);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                pa[s] = split_f2(geo[G_PAX + s]);
                u[s] = tf_mul(fq, split_f2(geo[G_PQX + s]));
                if constexpr (CB) pb[s] = tf_add(pa[s], split_f2(geo[G_ABX + s]));
            }
        }
        if constexpr (KET) {
            const F2 iq = split_f2(geo[G_IQ]), fp = split_f2(geo[G_P] * ipq);
            hiq = {0.5f * iq.h, 0.5f * iq.l};
            a01 = tf_mul(hiq, fp);
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                qc[s] = split_f2(geo[G_QCX + s]);
                nv[s] = tf_neg(tf_mul(fp, split_f2(geo[G_PQX + s])));
                if constexpr (CD) qd[s] = tf_add(qc[s], split_f2(geo[G_CDX + s]));
            }
        }
    }

    // B and C of the root with x = t^2 and weight w (the slots of phase_setup; slots the class
    // does not use are zero)
    __device__ __forceinline__ void root(double xd, double w, float *bc) const {
        bc[S_WZ] = pref * f64_to_f32(w);
#pragma unroll
        for (int f = S_B00; f < S_WZ; ++f) bc[f] = 0.0f;
        if constexpr (BRA || KET) {
            const F2 x = split_f2(xd);
            if constexpr (BRA && KET) bc[S_B00] = hq * x.h;
            if constexpr (BRA) {
                bc[S_B10] = tf_fms(hip, a10, x);
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    bc[S_C0X + s] = tf_fms(pa[s], u[s], x);
                    if constexpr (CB) bc[C::S_CB + s] = tf_fms(pb[s], u[s], x);
                }
            }
            if constexpr (KET) {
                bc[S_B01] = tf_fms(hiq, a01, x);
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    bc[S_C1X + s] = tf_fms(qc[s], nv[s], x);
                    if constexpr (CD) bc[C::S_CD + s] = tf_fms(qd[s], nv[s], x);
                }
            }
        }
    }
};

// Root mu of the quartet (Boys F_0 alone for L = 0), mixed evaluation, as in phase_setup.
template <class C>
__device__ __forceinline__ void root_mixed(const Tables &tb, double T, int mu, double &x, double &w) {
    if constexpr (C::NAB + C::NCD == 0) {
        double F0, F1;
        boys_f01_mixed<false>(T, tb.boys_t01, tb.boys_t01_f, F0, F1);
        w = F0;
        x = 0.0;
    } else {
        rys_root<true>(tb, C::NRYS, mu, T, x, w);
    }
}

// Bra HRR (Eq. 7) of one VRR column g(e) (fixed k) into h[i][j], i <= La, j <= Lb.
// Built on A (swab = false): (i, j+1) = (i+1, j) + AB (i, j), i.e. transfer to b.
// Built on B (swab = true):  (i+1, j) = (i, j+1) + BA (i, j), i.e. transfer to a.
// Transferring away from the centre nearer to P keeps the cancellation factor of the transfer
// bounded (|AB| / |P - target| <= 2 for each step).
template <class C>
__device__ __forceinline__ void bra_hrr(const typename C::R (&g)[C::NAB + 1], typename C::R ab,
                                        bool swab, typename C::R (&h)[C::La + 1][C::Lb + 1]) {
    using R = typename C::R;
    if (!swab) {
        R t[C::Lb + 1][C::NAB + 1];
#pragma unroll
        for (int e = 0; e <= C::NAB; ++e) t[0][e] = g[e];
#pragma unroll
        for (int j = 1; j <= C::Lb; ++j)
#pragma unroll
            for (int e = 0; e + j <= C::NAB; ++e) t[j][e] = fma(ab, t[j - 1][e], t[j - 1][e + 1]);
#pragma unroll
        for (int i = 0; i <= C::La; ++i)
#pragma unroll
            for (int j = 0; j <= C::Lb; ++j) h[i][j] = t[j][i];
    } else {
        R t[C::La + 1][C::NAB + 1];
#pragma unroll
        for (int e = 0; e <= C::NAB; ++e) t[0][e] = g[e];
#pragma unroll
        for (int i = 1; i <= C::La; ++i)
#pragma unroll
            for (int e = 0; e + i <= C::NAB; ++e) t[i][e] = fma(-ab, t[i - 1][e], t[i - 1][e + 1]);
#pragma unroll
        for (int i = 0; i <= C::La; ++i)
#pragma unroll
            for (int j = 0; j <= C::Lb; ++j) h[i][j] = t[i][j];
    }
}

// Ket HRR of one transferred column s(0..NCD) (fixed i, j) into o[k][l], k <= Lc, l <= Ld;
// transfer to d (swcd = false) or to c (swcd = true), as for the bra.
template <class C>
__device__ __forceinline__ void ket_hrr(const typename C::R (&s)[C::NCD + 1], typename C::R cd,
                                        bool swcd, typename C::R (&o)[C::Lc + 1][C::Ld + 1]) {
    using R = typename C::R;
    if (!swcd) {
        R t[C::Ld + 1][C::NCD + 1];
#pragma unroll
        for (int k = 0; k <= C::NCD; ++k) t[0][k] = s[k];
#pragma unroll
        for (int l = 1; l <= C::Ld; ++l)
#pragma unroll
            for (int k = 0; k + l <= C::NCD; ++k) t[l][k] = fma(cd, t[l - 1][k], t[l - 1][k + 1]);
#pragma unroll
        for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
            for (int l = 0; l <= C::Ld; ++l) o[k][l] = t[l][k];
    } else {
        R t[C::Lc + 1][C::NCD + 1];
#pragma unroll
        for (int k = 0; k <= C::NCD; ++k) t[0][k] = s[k];
#pragma unroll
        for (int c = 1; c <= C::Lc; ++c)
#pragma unroll
            for (int k = 0; k + c <= C::NCD; ++k) t[c][k] = fma(-cd, t[c - 1][k], t[c - 1][k + 1]);
#pragma unroll
        for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
            for (int l = 0; l <= C::Ld; ++l) o[k][l] = t[k][l];
    }
}

// I layout per quartet: [xi][mu][i][k][j][l] (the (j,l) block is contiguous for phase D).
template <class C>
__device__ __forceinline__ int i_index(int xi, int mu, int i, int k, int j, int l) {
    return (((xi * C::NRYS + mu) * (C::La + 1) + i) * (C::Lc + 1) + k) * C::JLP +
           j * (C::Ld + 1) + l;
}

// Phase B: VRR column by column in k, bra HRR of each column; writes H (or I when fused).
template <class C>
__device__ __forceinline__ void phase_vrr(const typename C::R *bc, const typename C::R *rg, int mu,
                                          int xi, typename C::R *Hq, typename C::R *Iq) {
    using R = typename C::R;
    const R *b = bc + mu * C::SN;
    R c00 = b[S_C0X + xi], c01 = b[S_C1X + xi];
    R b00 = b[S_B00], b10 = b[S_B10], b01 = b[S_B01];
    R ab = rg[RG_ABX + xi];
    const bool swab = rg[RG_SWAB] != (R)0;
    R prev[C::NAB + 1], cur[C::NAB + 1];
    // column k = 0: G(i+1, 0) = C00 G(i, 0) + i B10 G(i-1, 0)
    cur[0] = (xi == 2) ? b[S_WZ] : (R)1;
#pragma unroll
    for (int i = 0; i < C::NAB; ++i)
        cur[i + 1] = c00 * cur[i] + (i > 0 ? (R)i * b10 * cur[i - 1] : (R)0);
#pragma unroll
    for (int i = 0; i <= C::NAB; ++i) prev[i] = (R)0;
    R hk[C::La + 1][C::Lb + 1][C::NCD + 1];
#pragma unroll
    for (int k = 0; k <= C::NCD; ++k) {
        R h[C::La + 1][C::Lb + 1];
        bra_hrr<C>(cur, ab, swab, h);
        if constexpr (C::FUSE_BC) {
#pragma unroll
            for (int i = 0; i <= C::La; ++i)
#pragma unroll
                for (int j = 0; j <= C::Lb; ++j) hk[i][j][k] = h[i][j];
        } else {
#pragma unroll
            for (int i = 0; i <= C::La; ++i)
#pragma unroll
                for (int j = 0; j <= C::Lb; ++j)
                    Hq[(((xi * C::NRYS + mu) * (C::La + 1) + i) * (C::Lb + 1) + j) * (C::NCD + 1) +
                       k] = h[i][j];
        }
        if (k < C::NCD) {
            // G(i, k+1) = C00' G(i, k) + k B01 G(i, k-1) + i B00 G(i-1, k)
            R nxt[C::NAB + 1];
#pragma unroll
            for (int i = 0; i <= C::NAB; ++i) {
                R v = c01 * cur[i];
                if (k > 0) v = fma((R)k * b01, prev[i], v);
                if (i > 0) v = fma((R)i * b00, cur[i - 1], v);
                nxt[i] = v;
            }
#pragma unroll
            for (int i = 0; i <= C::NAB; ++i) {
                prev[i] = cur[i];
                cur[i] = nxt[i];
            }
        }
    }
    if constexpr (C::FUSE_BC) {
        R cd = rg[RG_CDX + xi];
        const bool swcd = rg[RG_SWCD] != (R)0;
#pragma unroll
        for (int i = 0; i <= C::La; ++i)
#pragma unroll
            for (int j = 0; j <= C::Lb; ++j) {
                R s[C::NCD + 1];
#pragma unroll
                for (int k = 0; k <= C::NCD; ++k) s[k] = hk[i][j][k];
                R o[C::Lc + 1][C::Ld + 1];
                ket_hrr<C>(s, cd, swcd, o);
#pragma unroll
                for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
                    for (int l = 0; l <= C::Ld; ++l) Iq[i_index<C>(xi, mu, i, k, j, l)] = o[k][l];
            }
    }
}

// Phase B of the four-index path (Cfg::DIRECT): the 2-D integrals I(i, j, k, l) of one
// (quartet, root, axis) by the Rys recursion in which every index is raised with the C
// coefficient of its own centre (the recurrences of the 2-D integrals behind Eqs. 6-7 before
// the transfer relation is introduced):
//   I(i+1, 0, 0, 0) = C00_A I(i) + i B10 I(i-1)
//   I(i, j+1, 0, 0) = C00_B I(i, j) + j B10 I(i, j-1) + i B10 I(i-1, j)
//   I(i, j, k+1, 0) = C00'_C I(k) + k B01 I(k-1) + (i I(i-1, j) + j I(i, j-1)) B00 at k
//   I(i, j, k, l+1) = C00'_D I(l) + l B01 I(l-1) + k B01 I(k-1, l) + (i I(i-1) + j I(j-1)) B00
// where C00_X = (P - X) - q x / (p+q) (P - Q), C00'_Y = (Q - Y) + p x / (p+q) (P - Q).
// Exact arithmetic gives the VRR + HRR values; in FP32 no step subtracts transferred
// values of a larger magnitude, so the rounding is not amplified.  The (i, j) plane of the
// current (k, l) is kept in registers, lower planes are read back from the I block already
// written (a small register footprint next to the accumulators of phase D).
template <class C>
__device__ __forceinline__ void phase_direct(const typename C::R *bc, int mu, int xi,
                                             typename C::R *Iq) {
    using R = typename C::R;
    constexpr int NI = C::La + 1, NJ = C::Lb + 1;
    const R *b = bc + mu * C::SN;
    const R cA = b[S_C0X + xi], cC = b[S_C1X + xi];
    R cB = (R)0, cD = (R)0;
    if constexpr (C::Lb > 0) cB = b[C::S_CB + xi];
    if constexpr (C::Ld > 0) cD = b[C::S_CD + xi];
    const R b00 = b[S_B00], b10 = b[S_B10], b01 = b[S_B01];
    R *blk = Iq + i_index<C>(xi, mu, 0, 0, 0, 0);
    // plane (k, l) = (0, 0)
    R pl[NI][NJ];
    pl[0][0] = (xi == 2) ? b[S_WZ] : (R)1;
#pragma unroll
    for (int i = 1; i < NI; ++i)
        pl[i][0] = i > 1 ? fma((R)(i - 1) * b10, pl[i - 2][0], cA * pl[i - 1][0]) : cA * pl[i - 1][0];
#pragma unroll
    for (int j = 1; j < NJ; ++j)
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            R v = cB * pl[i][j - 1];
            if (j > 1) v = fma((R)(j - 1) * b10, pl[i][j - 2], v);
            if (i > 0) v = fma((R)i * b10, pl[i - 1][j - 1], v);
            pl[i][j] = v;
        }
#pragma unroll
    for (int k = 0; k <= C::Lc; ++k) {
        if (k > 0) {
            // raise k at l = 0 from the planes (k-1, 0) and (k-2, 0) read back from the I block
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int e = (i * (C::Lc + 1) + k) * C::JLP + j * (C::Ld + 1);
                    R v = cC * blk[e - C::JLP];
                    if (k > 1) v = fma((R)(k - 1) * b01, blk[e - 2 * C::JLP], v);
                    if (i > 0) v = fma((R)i * b00, blk[e - (C::Lc + 2) * C::JLP], v);
                    if (j > 0) v = fma((R)j * b00, blk[e - C::JLP - (C::Ld + 1)], v);
                    pl[i][j] = v;
                }
        }
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j) blk[(i * (C::Lc + 1) + k) * C::JLP + j * (C::Ld + 1)] = pl[i][j];
        if constexpr (C::Ld > 0) {
            // raise l: the plane (k, l-1) stays in registers, (k, l-2) and (k-1, l-1) are read
            // back from the I block (keeps the register footprint at two planes)
            R q1[NI][NJ];
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) q1[i][j] = pl[i][j];
#pragma unroll
            for (int l = 1; l <= C::Ld; ++l) {
                R nw[NI][NJ];
#pragma unroll
                for (int i = 0; i < NI; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int e = (i * (C::Lc + 1) + k) * C::JLP + j * (C::Ld + 1) + l;
                        R v = cD * q1[i][j];
                        if (l > 1) v = fma((R)(l - 1) * b01, blk[e - 2], v);
                        if (k > 0) v = fma((R)k * b01, blk[e - C::JLP - 1], v);
                        if (i > 0) v = fma((R)i * b00, q1[i - 1][j], v);
                        if (j > 0) v = fma((R)j * b00, q1[i][j - 1], v);
                        nw[i][j] = v;
                    }
#pragma unroll
                for (int i = 0; i < NI; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        blk[(i * (C::Lc + 1) + k) * C::JLP + j * (C::Ld + 1) + l] = nw[i][j];
                        q1[i][j] = nw[i][j];
                    }
            }
        }
    }
}

// VRR + bra HRR + ket HRR of one (root, axis) entirely in registers: I[(i, k, j, l)] in the
// layout of i_index for fixed (xi, mu).  Used by the thread-per-quartet kernel.
template <class C>
__device__ __forceinline__ void axis_2d(const typename C::R *b, const typename C::R *rg, int xi,
                                        typename C::R (&I)[C::IBLK]) {
    using R = typename C::R;
    R c00 = b[S_C0X + xi], c01 = b[S_C1X + xi];
    R b00 = b[S_B00], b10 = b[S_B10], b01 = b[S_B01];
    R ab = rg[RG_ABX + xi], cd = rg[RG_CDX + xi];
    const bool swab = rg[RG_SWAB] != (R)0, swcd = rg[RG_SWCD] != (R)0;
    R prev[C::NAB + 1], cur[C::NAB + 1];
    cur[0] = (xi == 2) ? b[S_WZ] : (R)1;
#pragma unroll
    for (int i = 0; i < C::NAB; ++i)
        cur[i + 1] = c00 * cur[i] + (i > 0 ? (R)i * b10 * cur[i - 1] : (R)0);
#pragma unroll
    for (int i = 0; i <= C::NAB; ++i) prev[i] = (R)0;
    R hk[C::La + 1][C::Lb + 1][C::NCD + 1];
#pragma unroll
    for (int k = 0; k <= C::NCD; ++k) {
        R h[C::La + 1][C::Lb + 1];
        bra_hrr<C>(cur, ab, swab, h);
#pragma unroll
        for (int i = 0; i <= C::La; ++i)
#pragma unroll
            for (int j = 0; j <= C::Lb; ++j) hk[i][j][k] = h[i][j];
        if (k < C::NCD) {
            R nxt[C::NAB + 1];
#pragma unroll
            for (int i = 0; i <= C::NAB; ++i) {
                R v = c01 * cur[i];
                if (k > 0) v = fma((R)k * b01, prev[i], v);
                if (i > 0) v = fma((R)i * b00, cur[i - 1], v);
                nxt[i] = v;
            }
#pragma unroll
            for (int i = 0; i <= C::NAB; ++i) {
                prev[i] = cur[i];
                cur[i] = nxt[i];
            }
        }
    }
#pragma unroll
    for (int i = 0; i <= C::La; ++i)
#pragma unroll
        for (int j = 0; j <= C::Lb; ++j) {
            R sv[C::NCD + 1];
#pragma unroll
            for (int k = 0; k <= C::NCD; ++k) sv[k] = hk[i][j][k];
            R o[C::Lc + 1][C::Ld + 1];
            ket_hrr<C>(sv, cd, swcd, o);
#pragma unroll
            for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
                for (int l = 0; l <= C::Ld; ++l)
                    I[((i * (C::Lc + 1) + k) * (C::Lb + 1) + j) * (C::Ld + 1) + l] = o[k][l];
        }
}

// Phase C: ket HRR for one (mu, xi, i, j).
template <class C>
__device__ __forceinline__ void phase_ket(const typename C::R *rg, int mu, int xi, int i, int j,
                                          const typename C::R *Hq, typename C::R *Iq) {
    using R = typename C::R;
    R s[C::NCD + 1];
    const R *src = Hq + (((xi * C::NRYS + mu) * (C::La + 1) + i) * (C::Lb + 1) + j) * (C::NCD + 1);
#pragma unroll
    for (int k = 0; k <= C::NCD; ++k) s[k] = src[k];
    R o[C::Lc + 1][C::Ld + 1];
    ket_hrr<C>(s, rg[RG_CDX + xi], rg[RG_SWCD] != (R)0, o);
#pragma unroll
    for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
        for (int l = 0; l <= C::Ld; ++l) Iq[i_index<C>(xi, mu, i, k, j, l)] = o[k][l];
}

// Phase D for b-chunk CH: acc[bb][d] (+)= sum_mu X[bx][dx] Y[by][dy] Z[bz][dz], where X, Y, Z
// are the (j, l) blocks of I at (i, k) = (a_xi, c_xi) for xi = x, y, z.
template <class C, int CH, bool KAHAN>
__device__ __forceinline__ void quad_chunk(const typename C::R *Iq, int a, int c,
                                           typename C::R (&acc)[C::BCH][C::ND],
                                           typename C::R (&comp)[C::BCH][C::ND], bool first) {
    using R = typename C::R;
    constexpr int B0 = CH * C::BCH;
    constexpr int NBC = imin(C::BCH, C::NB - B0);
    constexpr int LD1 = C::Ld + 1;
    const int ax = c_cart[C::La][a][0], ay = c_cart[C::La][a][1], az = c_cart[C::La][a][2];
    const int cx = c_cart[C::Lc][c][0], cy = c_cart[C::Lc][c][1], cz = c_cart[C::Lc][c][2];
    R part[KAHAN ? C::BCH : 1][KAHAN ? C::ND : 1];
    if constexpr (KAHAN) {
#pragma unroll
        for (int bb = 0; bb < C::BCH; ++bb)
#pragma unroll
            for (int d = 0; d < C::ND; ++d) part[bb][d] = (R)0;
    } else if (first) {
#pragma unroll
        for (int bb = 0; bb < C::BCH; ++bb)
#pragma unroll
            for (int d = 0; d < C::ND; ++d) acc[bb][d] = (R)0;
    }
    const R *px = Iq + i_index<C>(0, 0, ax, cx, 0, 0);
    const R *py = Iq + i_index<C>(1, 0, ay, cy, 0, 0);
    const R *pz = Iq + i_index<C>(2, 0, az, cz, 0, 0);
    constexpr int MU_STRIDE = C::IBLKP;
#pragma unroll 1
    for (int mu = 0; mu < C::NRYS; ++mu) {
#pragma unroll
        for (int bb = 0; bb < NBC; ++bb) {
            constexpr int dummy = 0;
            (void)dummy;
            const int b = B0 + bb;
            const int bx = cart_x(C::Lb, b), by = cart_y(C::Lb, b), bz = cart_z(C::Lb, b);
            R X[LD1], Y[LD1], Z[LD1];
#pragma unroll
            for (int t = 0; t < LD1; ++t) {
                X[t] = px[bx * LD1 + t];
                Y[t] = py[by * LD1 + t];
                Z[t] = pz[bz * LD1 + t];
            }
#pragma unroll
            for (int d = 0; d < C::ND; ++d) {
                const int dx = cart_x(C::Ld, d), dy = cart_y(C::Ld, d), dz = cart_z(C::Ld, d);
                R xy = X[dx] * Y[dy];
                if constexpr (KAHAN)
                    part[bb][d] = fma(xy, Z[dz], part[bb][d]);
                else
                    acc[bb][d] = fma(xy, Z[dz], acc[bb][d]);
            }
        }
        px += MU_STRIDE;
        py += MU_STRIDE;
        pz += MU_STRIDE;
    }
    if constexpr (KAHAN) {
#pragma unroll
        for (int bb = 0; bb < C::BCH; ++bb)
#pragma unroll
            for (int d = 0; d < C::ND; ++d) {
                if (first) {
                    acc[bb][d] = part[bb][d];
                    comp[bb][d] = (R)0;
                } else {
                    // Kahan-compensated sum over primitive quartets
                    R y = part[bb][d] - comp[bb][d];
                    R t = acc[bb][d] + y;
                    comp[bb][d] = (t - acc[bb][d]) - y;
                    acc[bb][d] = t;
                }
            }
    }
}

template <class C, bool KAHAN>
__device__ __forceinline__ void quad_dispatch(int ch, const typename C::R *Iq, int a, int c,
                                              typename C::R (&acc)[C::BCH][C::ND],
                                              typename C::R (&comp)[C::BCH][C::ND], bool first) {
    if constexpr (C::NCH == 1) {
        quad_chunk<C, 0, KAHAN>(Iq, a, c, acc, comp, first);
    } else {
        switch (ch) {
            case 0: quad_chunk<C, 0, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 1: if constexpr (C::NCH > 1) quad_chunk<C, 1, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 2: if constexpr (C::NCH > 2) quad_chunk<C, 2, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 3: if constexpr (C::NCH > 3) quad_chunk<C, 3, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 4: if constexpr (C::NCH > 4) quad_chunk<C, 4, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 5: if constexpr (C::NCH > 5) quad_chunk<C, 5, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 6: if constexpr (C::NCH > 6) quad_chunk<C, 6, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 7: if constexpr (C::NCH > 7) quad_chunk<C, 7, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 8: if constexpr (C::NCH > 8) quad_chunk<C, 8, KAHAN>(Iq, a, c, acc, comp, first); break;
            case 9: if constexpr (C::NCH > 9) quad_chunk<C, 9, KAHAN>(Iq, a, c, acc, comp, first); break;
            default: break;
        }
    }
}

// ---------------------------------------------------------------------------------------
// One tile of Q quartets (tile index `tile`) of the phase kernel.  PRESET: phases A0/A1 were
// done by eri_setup_kernel and their results are read from args.setup.
template <class C, bool KAHAN, bool PRESET = false>
__device__ __forceinline__ void class_tile(const ShellsDev &sh, const Tables &tb,
                                           const ClassArgs &args, long long tile,
                                           unsigned char *smem) {
    using R = typename C::R;
    double *geo_s = reinterpret_cast<double *>(smem + C::OFF_GEO);
    R *rg_s = reinterpret_cast<R *>(smem + C::OFF_RG);
    R *bc_s = reinterpret_cast<R *>(smem + C::OFF_BC);
    unsigned long long *bmax_s = reinterpret_cast<unsigned long long *>(smem + C::OFF_BMAX);
    R *H_s = reinterpret_cast<R *>(smem + C::OFF_H);
    R *I_s = reinterpret_cast<R *>(smem + C::OFF_I);
    __shared__ int maxprim_s;

    const int tid = threadIdx.x;
    const long long q0 = tile * C::Q;
    const int qn = (int)((args.nq - q0) < C::Q ? (args.nq - q0) : C::Q);

    // phase D item of this thread (fixed across primitive iterations)
    const bool has_item = tid < C::Q * C::ITEMS_D;
    int dq = 0, da = 0, dc = 0, dch = 0;
    if (has_item) {
        dq = tid / C::ITEMS_D;
        int r = tid % C::ITEMS_D;
        da = r / (C::NC * C::NCH);
        dc = (r / C::NCH) % C::NC;
        dch = r % C::NCH;
    }
    R acc[C::BCH][C::ND];
    R comp[C::BCH][C::ND];  // Kahan compensation; eliminated when KAHAN is false

    if (tid == 0) maxprim_s = 1;
    __syncthreads();
    for (int prim = 0; prim < maxprim_s; ++prim) {
        if constexpr (PRESET) {
            // setup values of the tile, field-major in the setup buffer (coalesced loads)
            const R *su = reinterpret_cast<const R *>(args.setup) + q0;
            const int ss = (int)args.setup_stride;  // <= 2^20: 32-bit offsets
            for (int it = tid; it < C::Q * C::SETUP_GEO; it += C::THREADS) {
                int f = it / C::Q, q = it % C::Q;
                rg_s[q * RG_N + f] = q < qn ? su[f * ss + q] : (R)0;
            }
            for (int it = tid; it < C::Q * C::NRYS * C::SN; it += C::THREADS) {
                int f = it / C::Q, q = it % C::Q;
                bc_s[q * C::NRYS * C::SN + f] = q < qn ? su[(C::SETUP_GEO + f) * ss + q] : (R)0;
            }
            __syncthreads();
        } else {
            // A0: geometry per quartet (canonical shell order)
            for (int q = tid; q < C::Q; q += C::THREADS) {
                int np = 0;
                double *geo = geo_s + q * G_N;
                if (q < qn) {
                    int4 g = args.quartets[q0 + q];
                    int4 qt = make_int4(pick(g, args.perm[0]), pick(g, args.perm[1]),
                                        pick(g, args.perm[2]), pick(g, args.perm[3]));
                    geometry_of<C>(sh, args, qt, prim, geo, np);
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
            }
            __syncthreads();
            // A1: roots, weights, B and C per (quartet, root).  For primitive plans (no Kahan
            // sums) the mixed path forms B and C in two-float FP32 exactly as the split path's
            // setup kernel does (the persistent form of those plans then matches the per-class
            // launches bit for bit); contracted plans keep the FP64 formation, cheaper per item
            for (int it = tid; it < C::Q * C::NRYS; it += C::THREADS) {
                int q = it / C::NRYS, mu = it % C::NRYS;
                if constexpr (sizeof(R) == 4 && !KAHAN) {
                    const double *geo = geo_s + q * G_N;
                    SetupTF<C> pre;
                    pre.init(geo);
                    double x, w;
                    root_mixed<C>(tb, geo[G_T], mu, x, w);
                    pre.root(x, w, bc_s + (q * C::NRYS + mu) * C::SN);
                } else {
                    phase_setup<C>(tb, geo_s + q * G_N, mu, bc_s + (q * C::NRYS + mu) * C::SN);
                }
            }
            __syncthreads();
        }
        // B: VRR (+ bra HRR, + ket HRR when fused), or the four-index recursion, per
        // (quartet, root, axis)
        for (int it = tid; it < C::Q * C::NRYS * 3; it += C::THREADS) {
            int q = it / (C::NRYS * 3), r = it % (C::NRYS * 3);
            int mu = r / 3, xi = r % 3;
            if constexpr (C::DIRECT)
                phase_direct<C>(bc_s + q * C::NRYS * C::SN, mu, xi,
                                I_s + (size_t)q * (C::I_BYTES / sizeof(R)));
            else
                phase_vrr<C>(bc_s + q * C::NRYS * C::SN, rg_s + q * RG_N, mu, xi,
                             H_s + (size_t)q * (C::H_BYTES / sizeof(R)),
                             I_s + (size_t)q * (C::I_BYTES / sizeof(R)));
        }
        __syncthreads();
        if constexpr (!C::FUSE_BC && !C::DIRECT) {
            constexpr int NIJ = (C::La + 1) * (C::Lb + 1);
            for (int it = tid; it < C::Q * C::NRYS * 3 * NIJ; it += C::THREADS) {
                int q = it / (C::NRYS * 3 * NIJ), r = it % (C::NRYS * 3 * NIJ);
                int mu = r / (3 * NIJ);
                r %= 3 * NIJ;
                int xi = r / NIJ, ij = r % NIJ;
                phase_ket<C>(rg_s + q * RG_N, mu, xi, ij / (C::Lb + 1), ij % (C::Lb + 1),
                             H_s + (size_t)q * (C::H_BYTES / sizeof(R)),
                             I_s + (size_t)q * (C::I_BYTES / sizeof(R)));
            }
            __syncthreads();
        }
        // D: quadrature into register accumulators
        if (has_item)
            quad_dispatch<C, KAHAN>(dch, I_s + (size_t)dq * (C::I_BYTES / sizeof(R)), da, dc, acc,
                                    comp, prim == 0);
        __syncthreads();
    }

    const bool live = has_item && dq < qn;
    const int st0 = args.ostride[0], st1 = args.ostride[1], st2 = args.ostride[2],
              st3 = args.ostride[3];
    if (args.out_fp64 != nullptr) {
        // FP64 output in the generic class's row-major order
        if (live) {
            double *o = args.out_fp64 + (q0 + dq) * (long long)C::NERI + da * st0 + dc * st2;
            bool bad = false;
#pragma unroll
            for (int bb = 0; bb < C::BCH; ++bb) {
                int b = dch * C::BCH + bb;
                if (b < C::NB) {
#pragma unroll
                    for (int d = 0; d < C::ND; ++d) {
                        bad |= !RTraits<R>::finite(acc[bb][d]);
                        o[b * st1 + d * st3] = RTraits<R>::to_f64(acc[bb][d]);
                    }
                }
            }
            if (bad) atomicOr(args.err, 1);
        }
        return;
    }

    // ---- compressed output (Sec. II-D) ----
    for (int q = tid; q < C::Q; q += C::THREADS) bmax_s[q] = 0ull;
    __syncthreads();
    if (live) {
        // b_max = max |x| over the quartet; non-negative IEEE values order like their bit
        // patterns, so an integer atomicMax on the bits is exact.  Done in the accumulation
        // type: a conversion per value would occupy the (slow) FP64 pipe in mixed precision.
        bool bad = false;
        if constexpr (sizeof(R) == 8) {
            unsigned long long mb = 0ull;
#pragma unroll
            for (int bb = 0; bb < C::BCH; ++bb)
                if (dch * C::BCH + bb < C::NB)
#pragma unroll
                    for (int d = 0; d < C::ND; ++d) {
                        double v = fabs((double)acc[bb][d]);
                        bad |= !(v <= 1.7976931348623157e308);
                        unsigned long long u = (unsigned long long)__double_as_longlong(v);
                        mb = u > mb ? u : mb;
                    }
            atomicMax(bmax_s + dq, mb);
        } else {
            unsigned int mb = 0u;
#pragma unroll
            for (int bb = 0; bb < C::BCH; ++bb)
                if (dch * C::BCH + bb < C::NB)
#pragma unroll
                    for (int d = 0; d < C::ND; ++d) {
                        unsigned int u = __float_as_uint((float)acc[bb][d]) & 0x7fffffffu;
                        bad |= u >= 0x7f800000u;  // inf or nan
                        mb = u > mb ? u : mb;
                    }
            atomicMax(reinterpret_cast<unsigned int *>(bmax_s + dq), mb);
        }
        if (bad) atomicOr(args.err, 1);
    }
    // staging buffer for the tile's bitstream (aliases the H/I region)
    const int bits = args.bits;
    const long long bit0 = q0 * (long long)C::NERI * bits;
    const long long bit1 = (q0 + qn) * (long long)C::NERI * bits;
    const long long w0 = bit0 >> 5;
    const long long w1 = (bit1 + 31) >> 5;
    const int nw = (int)(w1 - w0);
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + C::OFF_U);
    __syncthreads();  // quadrature reads of I are complete; b_max final
    for (int w = tid; w < nw; w += C::THREADS) stage[w] = 0u;
    __syncthreads();
    if (live) {
        // eps = b_max / M rounded to FP32 (Eq. 9).  In mixed precision b_max is an FP32 value and
        // M is exact in FP32, so the correctly rounded FP32 quotient is that rounding.
        float eps;
        R inv;
        if constexpr (sizeof(R) == 8) {
            const double M = (double)((1u << (bits - 1)) - 1u);
            eps = (float)(__longlong_as_double((long long)bmax_s[dq]) / M);
            inv = (eps > 0.0f) ? (R)(1.0 / (double)eps) : (R)0;
        } else {
            const float M = (float)((1u << (bits - 1)) - 1u);
            eps = __uint_as_float(*reinterpret_cast<const unsigned int *>(bmax_s + dq)) / M;
            inv = (eps > 0.0f) ? (R)(1.0f / eps) : (R)0;
        }
        if (da == 0 && dc == 0 && dch == 0) args.scales[q0 + dq] = eps;
        const uint32_t mask = (1u << bits) - 1u;
        const R Mr = (R)((1u << (bits - 1)) - 1u);
        // bit offsets relative to the tile's first stage word, in 32-bit arithmetic (the tile
        // holds at most Q * n_ERIQ * bits < 2^31 bits)
        const int head = (int)(bit0 & 31);
        const int qbase = dq * C::NERI + da * st0 + dc * st2;
        // byte widths: every code owns its byte / halfword of the stage, so a plain store
        // replaces the shared-memory atomics of the generic bit packing
        uint16_t *st16 = reinterpret_cast<uint16_t *>(stage) + (head >> 4);
        uint8_t *st8 = reinterpret_cast<uint8_t *>(stage) + (head >> 3);
#pragma unroll
        for (int bb = 0; bb < C::BCH; ++bb) {
            int b = dch * C::BCH + bb;
            if (b < C::NB) {
#pragma unroll
                for (int d = 0; d < C::ND; ++d) {
                    R v = RTraits<R>::round_away(acc[bb][d] * inv);
                    v = v > Mr ? Mr : (v < -Mr ? -Mr : v);
                    uint32_t code = to_code<R>(v, bits) & mask;
                    const int e = qbase + b * st1 + d * st3;
                    if (bits == 16) {
                        st16[e] = (uint16_t)code;
                    } else if (bits == 8) {
                        st8[e] = (uint8_t)code;
                    } else {
                        const int s = head + e * bits;
                        int wi = s >> 5, off = s & 31;
                        atomicOr(stage + wi, code << off);
                        if (off + bits > 32) atomicOr(stage + wi + 1, code >> (32 - off));
                    }
                }
            }
        }
    }
    __syncthreads();
    // store the tile's words; partial edge words are merged with the neighbour tile's bits
    const bool last_tile = (q0 + qn) >= args.nq;
    const int head_bits = (int)(bit0 & 31);
    const int tail_bits = (int)(bit1 & 31);
    for (int w = tid; w < nw; w += C::THREADS) {
        uint32_t v = stage[w];
        long long gw = w0 + w;
        uint32_t keep = 0xffffffffu;  // bits of this word owned by this tile
        if (w == 0 && head_bits) keep &= ~((1u << head_bits) - 1u);
        if (w == nw - 1 && tail_bits && !last_tile) keep &= (1u << tail_bits) - 1u;
        if (keep == 0xffffffffu) {
            args.packed[gw] = v;
        } else {
            atomicAnd(args.packed + gw, ~keep);
            atomicOr(args.packed + gw, v & keep);
        }
    }
    if (last_tile) {
        for (long long w = w1 + tid; w < args.seg_words; w += C::THREADS) args.packed[w] = 0u;
    }
}

template <class C, bool KAHAN, bool PRESET = false>
__global__ void __launch_bounds__(C::THREADS)
eri_class_kernel(ShellsDev sh, Tables tb, ClassArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    class_tile<C, KAHAN, PRESET>(sh, tb, args, blockIdx.x, smem);
}

// Setup stage of the split path (primitive quartets, K = 1): one thread per quartet computes
// the Gaussian-product geometry, the Rys roots and weights and the B, C arrays in FP64 and
// stores them (type R) field-major, so that every thread of this kernel does FP64 work and
// the recurrence kernel that follows does none.
template <class C>
__global__ void __launch_bounds__(128)
eri_setup_kernel(ShellsDev sh, Tables tb, ClassArgs args, typename C::R *out, long long stride) {
    using R = typename C::R;
    const long long q = (long long)blockIdx.x * 128 + threadIdx.x;
    if (q >= args.nq) return;
    const int st = (int)stride;  // <= 2^20: field offsets in 32-bit arithmetic
    int4 g = args.quartets[q];
    int4 qt = make_int4(pick(g, args.perm[0]), pick(g, args.perm[1]), pick(g, args.perm[2]),
                        pick(g, args.perm[3]));
    double geo[G_N];
    int np = 0;
    geometry_of<C>(sh, args, qt, 0, geo, np);
    R *o = out + q;
    o[0 * st] = to_r<R>(geo[G_ABX]);
    o[1 * st] = to_r<R>(geo[G_ABY]);
    o[2 * st] = to_r<R>(geo[G_ABZ]);
    o[3 * st] = to_r<R>(geo[G_CDX]);
    o[4 * st] = to_r<R>(geo[G_CDY]);
    o[5 * st] = to_r<R>(geo[G_CDZ]);
    o[6 * st] = to_r<R>(geo[G_SWAB]);
    o[7 * st] = to_r<R>(geo[G_SWCD]);
    if constexpr (sizeof(R) == 4) {
        SetupTF<C> pre;
        pre.init(geo);
#pragma unroll 1
        for (int mu = 0; mu < C::NRYS; ++mu) {
            double x, w;
            root_mixed<C>(tb, geo[G_T], mu, x, w);
            float bc[C::SN];
            pre.root(x, w, bc);
#pragma unroll
            for (int f = 0; f < C::SN; ++f) o[(C::SETUP_GEO + mu * C::SN + f) * st] = bc[f];
        }
    } else {
#pragma unroll 1
        for (int mu = 0; mu < C::NRYS; ++mu) {
            R bc[C::SN];
            phase_setup<C>(tb, geo, mu, bc);
#pragma unroll
            for (int f = 0; f < C::SN; ++f) o[(C::SETUP_GEO + mu * C::SN + f) * st] = bc[f];
        }
    }
}

// Persistent form: a grid sized to the resident CTAs pulls tiles from a work counter
// (atomicAdd, no waiting) until the class is exhausted; quartets of uneven contraction
// degree therefore balance dynamically.  The counter must be zero at launch.
template <class C, bool KAHAN>
__global__ void __launch_bounds__(C::THREADS)
eri_class_persistent(ShellsDev sh, Tables tb, ClassArgs args, unsigned long long *counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long tile_s;
    const long long n_tiles = (args.nq + C::Q - 1) / C::Q;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) tile_s = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long t = tile_s;
        if (t >= n_tiles) break;
        class_tile<C, KAHAN>(sh, tb, args, t, smem);
    }
}

// The four-index recursion of phase_direct for one (root, axis) in registers, in the layout of
// axis_2d (I[((i * (Lc+1) + k) * (Lb+1) + j) * (Ld+1) + l]); thread-per-quartet kernels.
template <class C>
__device__ __forceinline__ void axis_direct(const typename C::R *b, int xi,
                                            typename C::R (&I)[C::IBLK]) {
    using R = typename C::R;
    constexpr int LB1 = C::Lb + 1, LC1 = C::Lc + 1, LD1 = C::Ld + 1;
#define ERI_IX(i, k, j, l) ((((i) * LC1 + (k)) * LB1 + (j)) * LD1 + (l))
    const R cA = b[S_C0X + xi], cC = b[S_C1X + xi];
    R cB = (R)0, cD = (R)0;
    if constexpr (C::Lb > 0) cB = b[C::S_CB + xi];
    if constexpr (C::Ld > 0) cD = b[C::S_CD + xi];
    const R b00 = b[S_B00], b10 = b[S_B10], b01 = b[S_B01];
    I[0] = (xi == 2) ? b[S_WZ] : (R)1;
#pragma unroll
    for (int i = 1; i <= C::La; ++i) {
        R v = cA * I[ERI_IX(i - 1, 0, 0, 0)];
        if (i > 1) v = fma((R)(i - 1) * b10, I[ERI_IX(i - 2, 0, 0, 0)], v);
        I[ERI_IX(i, 0, 0, 0)] = v;
    }
#pragma unroll
    for (int j = 1; j <= C::Lb; ++j)
#pragma unroll
        for (int i = 0; i <= C::La; ++i) {
            R v = cB * I[ERI_IX(i, 0, j - 1, 0)];
            if (j > 1) v = fma((R)(j - 1) * b10, I[ERI_IX(i, 0, j - 2, 0)], v);
            if (i > 0) v = fma((R)i * b10, I[ERI_IX(i - 1, 0, j - 1, 0)], v);
            I[ERI_IX(i, 0, j, 0)] = v;
        }
#pragma unroll
    for (int k = 1; k <= C::Lc; ++k)
#pragma unroll
        for (int i = 0; i <= C::La; ++i)
#pragma unroll
            for (int j = 0; j <= C::Lb; ++j) {
                R v = cC * I[ERI_IX(i, k - 1, j, 0)];
                if (k > 1) v = fma((R)(k - 1) * b01, I[ERI_IX(i, k - 2, j, 0)], v);
                if (i > 0) v = fma((R)i * b00, I[ERI_IX(i - 1, k - 1, j, 0)], v);
                if (j > 0) v = fma((R)j * b00, I[ERI_IX(i, k - 1, j - 1, 0)], v);
                I[ERI_IX(i, k, j, 0)] = v;
            }
#pragma unroll
    for (int k = 0; k <= C::Lc; ++k)
#pragma unroll
        for (int l = 1; l <= C::Ld; ++l)
#pragma unroll
            for (int i = 0; i <= C::La; ++i)
#pragma unroll
                for (int j = 0; j <= C::Lb; ++j) {
                    R v = cD * I[ERI_IX(i, k, j, l - 1)];
                    if (l > 1) v = fma((R)(l - 1) * b01, I[ERI_IX(i, k, j, l - 2)], v);
                    if (k > 0) v = fma((R)k * b01, I[ERI_IX(i, k - 1, j, l - 1)], v);
                    if (i > 0) v = fma((R)i * b00, I[ERI_IX(i - 1, k, j, l - 1)], v);
                    if (j > 0) v = fma((R)j * b00, I[ERI_IX(i, k, j - 1, l - 1)], v);
                    I[ERI_IX(i, k, j, l)] = v;
                }
#undef ERI_IX
}

// ---------------------------------------------------------------------------------------
// Thread-per-quartet kernel for the small classes: each thread runs every stage of one
// quartet in registers (no shared-memory phases, no barriers before the store), so the FP64
// setup of all threads overlaps.  Shared memory is used only to pack the compressed tile.
// PRESET: the geometry and per-root setup come from the setup kernel's records (FP32 only).

// 2-D integrals of one root and the quadrature (Eq. 8) into the thread's accumulators.
template <class C>
__device__ __forceinline__ void tpq_root(const typename C::R *bc, const typename C::R *rg,
                                         typename C::R (&acc)[C::NERI]) {
    using R = typename C::R;
    R X[C::IBLK], Y[C::IBLK], Z[C::IBLK];
    if constexpr (C::DIRECT) {
        axis_direct<C>(bc, 0, X);
        axis_direct<C>(bc, 1, Y);
        axis_direct<C>(bc, 2, Z);
    } else {
        axis_2d<C>(bc, rg, 0, X);
        axis_2d<C>(bc, rg, 1, Y);
        axis_2d<C>(bc, rg, 2, Z);
    }
#pragma unroll
    for (int a = 0; a < C::NA; ++a)
#pragma unroll
        for (int b = 0; b < C::NB; ++b)
#pragma unroll
            for (int c = 0; c < C::NC; ++c)
#pragma unroll
                for (int d = 0; d < C::ND; ++d) {
                    constexpr int LB1 = C::Lb + 1, LC1 = C::Lc + 1, LD1 = C::Ld + 1;
                    const int ix = ((cart_x(C::La, a) * LC1 + cart_x(C::Lc, c)) * LB1 + cart_x(C::Lb, b)) * LD1 + cart_x(C::Ld, d);
                    const int iy = ((cart_y(C::La, a) * LC1 + cart_y(C::Lc, c)) * LB1 + cart_y(C::Lb, b)) * LD1 + cart_y(C::Ld, d);
                    const int iz = ((cart_z(C::La, a) * LC1 + cart_z(C::Lc, c)) * LB1 + cart_z(C::Lb, b)) * LD1 + cart_z(C::Ld, d);
                    const int o = ((a * C::NB + b) * C::NC + c) * C::ND + d;
                    acc[o] = fma(X[ix] * Y[iy], Z[iz], acc[o]);
                }
}

template <class C, bool PRESET = false>
__device__ __forceinline__ void tpq_tile(const ShellsDev &sh, const Tables &tb,
                                         const ClassArgs &args, long long tile,
                                         unsigned char *smem) {
    using R = typename C::R;
    const int tid = threadIdx.x;
    const long long q0 = tile * C::TPQ_THREADS;
    const int qn = (int)((args.nq - q0) < C::TPQ_THREADS ? (args.nq - q0) : C::TPQ_THREADS);
    const bool live = tid < qn;
    R acc[C::NERI];
#pragma unroll
    for (int o = 0; o < C::NERI; ++o) acc[o] = (R)0;
    if (live) {
        if constexpr (PRESET) {
            // field-major setup records: consecutive threads read consecutive words
            const R *su = reinterpret_cast<const R *>(args.setup) + (q0 + tid);
            const int ss = (int)args.setup_stride;  // <= 2^20: 32-bit offsets
            R rg[RG_N];
#pragma unroll
            for (int f = 0; f < RG_N; ++f) rg[f] = su[f * ss];
#pragma unroll 1
            for (int mu = 0; mu < C::NRYS; ++mu) {
                R bc[C::SN];
#pragma unroll
                for (int f = 0; f < C::SN; ++f) bc[f] = su[(C::SETUP_GEO + mu * C::SN + f) * ss];
                tpq_root<C>(bc, rg, acc);
            }
        } else {
            int4 g = args.quartets[q0 + tid];
            int4 qt = make_int4(pick(g, args.perm[0]), pick(g, args.perm[1]), pick(g, args.perm[2]),
                                pick(g, args.perm[3]));
            int nprim = 1;
            for (int prim = 0; prim < nprim; ++prim) {
                double geo[G_N];
                geometry_of<C>(sh, args, qt, prim, geo, nprim);
                R rg[RG_N];
#pragma unroll
                for (int x = 0; x < 3; ++x) {
                    rg[RG_ABX + x] = to_r<R>(geo[G_ABX + x]);
                    rg[RG_CDX + x] = to_r<R>(geo[G_CDX + x]);
                }
                rg[RG_SWAB] = to_r<R>(geo[G_SWAB]);
                rg[RG_SWCD] = to_r<R>(geo[G_SWCD]);
                if constexpr (C::SETUP_TF) {
                    SetupTF<C> pre;
                    pre.init(geo);
#pragma unroll 1
                    for (int mu = 0; mu < C::NRYS; ++mu) {
                        double x, w;
                        root_mixed<C>(tb, geo[G_T], mu, x, w);
                        R bc[C::SN];
                        pre.root(x, w, bc);
                        tpq_root<C>(bc, rg, acc);
                    }
                } else {
#pragma unroll 1
                    for (int mu = 0; mu < C::NRYS; ++mu) {
                        R bc[C::SN];
                        phase_setup<C>(tb, geo, mu, bc);
                        tpq_root<C>(bc, rg, acc);
                    }
                }
            }
        }
    }
    const int st0 = args.ostride[0], st1 = args.ostride[1], st2 = args.ostride[2],
              st3 = args.ostride[3];
    if (args.out_fp64 != nullptr) {
        if (live) {
            double *out = args.out_fp64 + (q0 + tid) * (long long)C::NERI;
            bool bad = false;
#pragma unroll
            for (int a = 0; a < C::NA; ++a)
#pragma unroll
                for (int b = 0; b < C::NB; ++b)
#pragma unroll
                    for (int c = 0; c < C::NC; ++c)
#pragma unroll
                        for (int d = 0; d < C::ND; ++d) {
                            const R v = acc[((a * C::NB + b) * C::NC + c) * C::ND + d];
                            bad |= !RTraits<R>::finite(v);
                            out[a * st0 + b * st1 + c * st2 + d * st3] = RTraits<R>::to_f64(v);
                        }
            if (bad) atomicOr(args.err, 1);
        }
        return;
    }
    // ---- compressed output (Sec. II-D) ----
    const int bits = args.bits;
    const long long bit0 = q0 * (long long)C::NERI * bits;
    const long long bit1 = (q0 + qn) * (long long)C::NERI * bits;
    const long long w0 = bit0 >> 5;
    const long long w1 = (bit1 + 31) >> 5;
    const int nw = (int)(w1 - w0);
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem);
    for (int w = tid; w < nw; w += C::TPQ_THREADS) stage[w] = 0u;
    __syncthreads();
    if (live) {
        R m = (R)0;
        bool bad = false;
#pragma unroll
        for (int o = 0; o < C::NERI; ++o) {
            R v = acc[o] < (R)0 ? -acc[o] : acc[o];
            bad |= !(v <= (R)3.0e38);
            m = v > m ? v : m;
        }
        if (bad) atomicOr(args.err, 1);
        float eps;
        R inv;
        if constexpr (sizeof(R) == 8) {
            const double M = (double)((1u << (bits - 1)) - 1u);
            eps = (float)((double)m / M);
            inv = (eps > 0.0f) ? (R)(1.0 / (double)eps) : (R)0;
        } else {
            eps = (float)m / (float)((1u << (bits - 1)) - 1u);
            inv = (eps > 0.0f) ? (R)(1.0f / eps) : (R)0;
        }
        args.scales[q0 + tid] = eps;
        const uint32_t mask = (1u << bits) - 1u;
        const R Mr = (R)((1u << (bits - 1)) - 1u);
        // bit offsets relative to the tile's first stage word, in 32-bit arithmetic
        const int head = (int)(bit0 & 31);
        const int tbase = tid * C::NERI;
        // byte widths: plain byte / halfword stores (each code owns its slot), else bit packing
        uint16_t *st16 = reinterpret_cast<uint16_t *>(stage) + (head >> 4);
        uint8_t *st8 = reinterpret_cast<uint8_t *>(stage) + (head >> 3);
#pragma unroll
        for (int a = 0; a < C::NA; ++a)
#pragma unroll
            for (int b = 0; b < C::NB; ++b)
#pragma unroll
                for (int c = 0; c < C::NC; ++c)
#pragma unroll
                    for (int d = 0; d < C::ND; ++d) {
                        R v = RTraits<R>::round_away(acc[((a * C::NB + b) * C::NC + c) * C::ND + d] * inv);
                        v = v > Mr ? Mr : (v < -Mr ? -Mr : v);
                        uint32_t code = to_code<R>(v, bits) & mask;
                        const int e = tbase + a * st0 + b * st1 + c * st2 + d * st3;
                        if (bits == 16) {
                            st16[e] = (uint16_t)code;
                        } else if (bits == 8) {
                            st8[e] = (uint8_t)code;
                        } else {
                            const int sb = head + e * bits;
                            int wi = sb >> 5, off = sb & 31;
                            atomicOr(stage + wi, code << off);
                            if (off + bits > 32) atomicOr(stage + wi + 1, code >> (32 - off));
                        }
                    }
    }
    __syncthreads();
    const bool last_tile = (q0 + qn) >= args.nq;
    const int head_bits = (int)(bit0 & 31);
    const int tail_bits = (int)(bit1 & 31);
    for (int w = tid; w < nw; w += C::TPQ_THREADS) {
        uint32_t v = stage[w];
        long long gw = w0 + w;
        uint32_t keep = 0xffffffffu;
        if (w == 0 && head_bits) keep &= ~((1u << head_bits) - 1u);
        if (w == nw - 1 && tail_bits && !last_tile) keep &= (1u << tail_bits) - 1u;
        if (keep == 0xffffffffu) {
            args.packed[gw] = v;
        } else {
            atomicAnd(args.packed + gw, ~keep);
            atomicOr(args.packed + gw, v & keep);
        }
    }
    if (last_tile) {
        for (long long w = w1 + tid; w < args.seg_words; w += C::TPQ_THREADS) args.packed[w] = 0u;
    }
}

template <class C, bool PRESET = false>
__global__ void __launch_bounds__(C::TPQ_THREADS, C::TPQ_MINB)
eri_tpq_kernel(ShellsDev sh, Tables tb, ClassArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    tpq_tile<C, PRESET>(sh, tb, args, blockIdx.x, smem);
}

template <class C>
__global__ void __launch_bounds__(C::TPQ_THREADS, C::TPQ_MINB)
eri_tpq_persistent(ShellsDev sh, Tables tb, ClassArgs args, unsigned long long *counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long tile_s;
    const long long n_tiles = (args.nq + C::TPQ_THREADS - 1) / C::TPQ_THREADS;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) tile_s = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long t = tile_s;
        if (t >= n_tiles) break;
        tpq_tile<C>(sh, tb, args, t, smem);
    }
}

// Host-side launch helper for one canonical class.
//   o.force_phase  use the shared-memory phase kernel even where the thread-per-quartet
//                  kernel exists (autotuning)
//   o.counter      non-null: persistent launch pulling tiles from this zeroed counter with
//                  o.grid CTAs (o.grid <= 0: every resident CTA, from the occupancy API)
template <int La, int Lb, int Lc, int Ld, typename R, bool KAHAN>
cudaError_t launch_class(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                         cudaStream_t stream, const LaunchOpts &o) {
    using C = Cfg<La, Lb, Lc, Ld, R>;
    if (args.nq <= 0) return cudaSuccess;
    int sms = 0;
    if (o.counter) {
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
        if (e != cudaSuccess) return e;
    }
    if constexpr (C::TPQ && !KAHAN) {
        if (!o.force_phase) {
            size_t smem = 0;
            if (args.out_fp64 == nullptr)
                smem = ((size_t)C::TPQ_THREADS * C::NERI * args.bits + 31) / 32 * 4 + 16;
            long long tiles = (args.nq + C::TPQ_THREADS - 1) / C::TPQ_THREADS;
            if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
            if (!o.counter) {
                if constexpr (C::TPQ_SPLIT) {
                    if (o.scratch) {
                        // FP64 setup kernel, then the FP32 thread-per-quartet kernel
                        const long long stride = (args.nq + 31) / 32 * 32;
                        eri_setup_kernel<C><<<(unsigned)((args.nq + 127) / 128), 128, 0, stream>>>(
                            sh, tb, args, reinterpret_cast<R *>(o.scratch), stride);
                        cudaError_t e = cudaGetLastError();
                        if (e != cudaSuccess) return e;
                        ClassArgs a2 = args;
                        a2.setup = o.scratch;
                        a2.setup_stride = stride;
                        eri_tpq_kernel<C, true><<<(unsigned)tiles, C::TPQ_THREADS, smem, stream>>>(sh, tb, a2);
                        return cudaGetLastError();
                    }
                }
                eri_tpq_kernel<C><<<(unsigned)tiles, C::TPQ_THREADS, smem, stream>>>(sh, tb, args);
                return cudaGetLastError();
            }
            int per_sm = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, eri_tpq_persistent<C>, C::TPQ_THREADS, smem);
            if (e != cudaSuccess) return e;
            long long grid = o.grid > 0 ? o.grid : (long long)per_sm * sms;
            grid = grid < tiles ? grid : tiles;
            eri_tpq_persistent<C><<<(unsigned)grid, C::TPQ_THREADS, smem, stream>>>(sh, tb, args,
                                                                                     o.counter);
            return cudaGetLastError();
        }
    }
    if constexpr (!KAHAN) {
        if (o.scratch && !o.counter) {
            // split path: FP64 setup kernel, then the recurrence/quadrature kernel
            long long blocks = (args.nq + 127) / 128;
            if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
            const long long stride = (args.nq + 31) / 32 * 32;
            eri_setup_kernel<C><<<(unsigned)blocks, 128, 0, stream>>>(
                sh, tb, args, reinterpret_cast<R *>(o.scratch), stride);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            ClassArgs a2 = args;
            a2.setup = o.scratch;
            a2.setup_stride = stride;
            auto k2 = eri_class_kernel<C, false, true>;
            e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
            if (e != cudaSuccess) return e;
            long long tiles = (args.nq + C::Q - 1) / C::Q;
            k2<<<(unsigned)tiles, C::THREADS, C::SMEM, stream>>>(sh, tb, a2);
            return cudaGetLastError();
        }
    }
    auto kern = eri_class_kernel<C, KAHAN>;
    auto pkern = eri_class_persistent<C, KAHAN>;
    cudaError_t e = cudaFuncSetAttribute(o.counter ? (const void *)pkern : (const void *)kern,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    long long tiles = (args.nq + C::Q - 1) / C::Q;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (!o.counter) {
        kern<<<(unsigned)tiles, C::THREADS, C::SMEM, stream>>>(sh, tb, args);
        return cudaGetLastError();
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pkern, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    long long grid = o.grid > 0 ? o.grid : (long long)per_sm * sms;
    grid = grid < tiles ? grid : tiles;
    if (grid < 1) grid = 1;
    pkern<<<(unsigned)grid, C::THREADS, C::SMEM, stream>>>(sh, tb, args, o.counter);
    return cudaGetLastError();
}

// The 55 canonical classes (Sec. II-B, Eq. 3): La >= Lb, Lc >= Ld, n_ga n_gb >= n_gc n_gd.
__host__ __device__ constexpr int canonical_class(int idx) {
    int k = 0;
    for (int La = 0; La < 4; ++La)
        for (int Lb = 0; Lb <= La; ++Lb)
            for (int Lc = 0; Lc < 4; ++Lc)
                for (int Ld = 0; Ld <= Lc; ++Ld)
                    if (ncart(La) * ncart(Lb) >= ncart(Lc) * ncart(Ld)) {
                        if (k == idx) return ((La * 4 + Lb) * 4 + Lc) * 4 + Ld;
                        ++k;
                    }
    return -1;
}
constexpr int kNumCanonical = 55;

}  // namespace eri
