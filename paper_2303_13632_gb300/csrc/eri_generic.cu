// eri_generic.cu -- ERIs of the classes with a g shell (L = 4) by one kernel whose angular
// momenta are run-time values.
//
// The per-class kernels of eri_kernels.cuh are specialised for each canonical class: every loop
// over components is unrolled and the intermediates live in registers.  For the 65 canonical
// classes with a g shell that specialisation would take the library build from minutes to the
// better part of an hour ([gg|gg] alone compiles for more than seven minutes in three variants),
// so these classes share one kernel per precision with the same stages of Sec. II-C in run-time
// loops over shared memory:
//   A0 geometry and prefactor        one thread per quartet (FP64, as the specialised kernels)
//   A1 Rys root/weight, B and C      one thread per (quartet, root) (FP64, rounded to R)
//   B  2-D integrals I(i, j, k, l)   one thread per (quartet, root, axis): the four-index Rys
//                                    recursion in which every index is raised with the C value of
//                                    its own centre (the recurrences behind Eqs. 6-7 before the
//                                    transfer relation; exact arithmetic gives the VRR + HRR values)
//   D  quadrature (Eq. 8)            one thread per (quartet, output), summed over the roots in R
//                                    and over primitives in FP64 (in the output or the scratch)
// Compressed output (Sec. II-D) then takes two more launches over the FP64 values: b_max and eps
// per quartet (Eq. 9), and the codes (Eq. 10) packed one output word per thread.
#include <algorithm>

#include "eri_internal.h"
#include "eri_kernels.cuh"

namespace eri {

namespace {

constexpr int kGenThreads = 256;
// B, C values per (quartet, root): the slots of phase_setup plus C00 relative to B and C00'
// relative to D
constexpr int kGenCB = S_N, kGenCD = S_N + 3, kGenSN = S_N + 6;

// geometry without the choice of transfer direction (the four-index recursion needs none)
struct GenGeo {
    static constexpr bool SWAB_OK = false, SWCD_OK = false;
};

struct GenShape {
    int L[4];        // canonical angular momenta
    int n[4];        // Cartesian components per shell
    int nrys, neri;  // roots, ERIs per quartet
    int iblk;        // 2-D integrals per (root, axis): (La+1)(Lb+1)(Lc+1)(Ld+1)
    int q;           // quartets per CTA
    int bc_off, i_off, smem;  // dynamic shared memory layout (bytes)
};

template <typename R>
GenShape gen_shape(const int L[4]) {
    GenShape g{};
    for (int k = 0; k < 4; ++k) {
        g.L[k] = L[k];
        g.n[k] = ncart(L[k]);
    }
    g.nrys = (L[0] + L[1] + L[2] + L[3]) / 2 + 1;
    g.neri = g.n[0] * g.n[1] * g.n[2] * g.n[3];
    g.iblk = (L[0] + 1) * (L[1] + 1) * (L[2] + 1) * (L[3] + 1);
    const int geo = G_N * 8, bc = g.nrys * kGenSN * (int)sizeof(R), ib = 3 * g.nrys * g.iblk * (int)sizeof(R);
    const int perq = geo + bc + ib + 16;
    g.q = std::max(1, std::min(64, (96 * 1024) / perq));
    g.bc_off = g.q * geo;
    g.i_off = ((g.bc_off + g.q * bc + 15) / 16) * 16;
    g.smem = g.i_off + g.q * ib;
    return g;
}

template <typename R>
__global__ void __launch_bounds__(kGenThreads)
eri_generic_kernel(ShellsDev sh, Tables tb, ClassArgs args, GenShape g, double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *geo_s = reinterpret_cast<double *>(smem);
    R *bc_s = reinterpret_cast<R *>(smem + g.bc_off);
    R *I_s = reinterpret_cast<R *>(smem + g.i_off);
    __shared__ int maxprim_s;
    const int tid = threadIdx.x;
    const long long q0 = (long long)blockIdx.x * g.q;
    const int qn = (int)((args.nq - q0) < g.q ? (args.nq - q0) : g.q);
    const int La = g.L[0], Lb = g.L[1], Lc = g.L[2], Ld = g.L[3];
    // strides of I(i, j, k, l) within one (root, axis) block
    const int sk = Ld + 1, sj = (Lc + 1) * sk, si = (Lb + 1) * sj;
    if (tid == 0) maxprim_s = 1;
    __syncthreads();
    for (int prim = 0; prim < maxprim_s; ++prim) {
        // A0: geometry of primitive quartet `prim` of each quartet
        for (int q = tid; q < g.q; q += kGenThreads) {
            double *geo = geo_s + q * G_N;
            int np = 0;
            if (q < qn) {
                const int4 gq = args.quartets[q0 + q];
                const int4 qt = make_int4(pick(gq, args.perm[0]), pick(gq, args.perm[1]),
                                          pick(gq, args.perm[2]), pick(gq, args.perm[3]));
                geometry_of<GenGeo>(sh, args, qt, prim, geo, np);
            } else {
                geo[G_PREF] = 0.0;
                geo[G_T] = 0.0;
                for (int s = G_P; s < G_N; ++s)
                    geo[s] = (s == G_P || s == G_Q || s == G_IP || s == G_IQ) ? 1.0 : (s == G_IPQ ? 0.5 : 0.0);
            }
            if (prim == 0 && np > 1) atomicMax(&maxprim_s, np);
        }
        __syncthreads();
        // A1: root and weight, B and C of each (quartet, root)
        for (int it = tid; it < g.q * g.nrys; it += kGenThreads) {
            const int q = it / g.nrys, mu = it - q * g.nrys;
            const double *geo = geo_s + q * G_N;
            double x, w;
            rys_root<sizeof(R) == 4>(tb, g.nrys, mu, geo[G_T], x, w);
            R *b = bc_s + (size_t)it * kGenSN;
            const double ipq = geo[G_IPQ];
            const double fq = geo[G_Q] * x * ipq, fp = geo[G_P] * x * ipq;
            b[S_B00] = to_r<R>(0.5 * x * ipq);
            b[S_B10] = to_r<R>((1.0 - fq) * (0.5 * geo[G_IP]));
            b[S_B01] = to_r<R>((1.0 - fp) * (0.5 * geo[G_IQ]));
            for (int s = 0; s < 3; ++s) {
                const double pq = geo[G_PQX + s];
                b[S_C0X + s] = to_r<R>(geo[G_PAX + s] - fq * pq);
                b[kGenCB + s] = to_r<R>((geo[G_PAX + s] + geo[G_ABX + s]) - fq * pq);
                b[S_C1X + s] = to_r<R>(geo[G_QCX + s] + fp * pq);
                b[kGenCD + s] = to_r<R>((geo[G_QCX + s] + geo[G_CDX + s]) + fp * pq);
            }
            b[S_WZ] = to_r<R>(geo[G_PREF] * w);
        }
        __syncthreads();
        // B: I(i, j, k, l) of each (quartet, root, axis), every index raised with its own centre
        for (int it = tid; it < g.q * g.nrys * 3; it += kGenThreads) {
            const int q = it / (g.nrys * 3), r = it - q * g.nrys * 3;
            const int mu = r / 3, xi = r - mu * 3;
            const R *b = bc_s + (size_t)(q * g.nrys + mu) * kGenSN;
            R *I = I_s + ((size_t)(q * 3 + xi) * g.nrys + mu) * g.iblk;
            const R cA = b[S_C0X + xi], cB = b[kGenCB + xi], cC = b[S_C1X + xi], cD = b[kGenCD + xi];
            const R b00 = b[S_B00], b10 = b[S_B10], b01 = b[S_B01];
            I[0] = xi == 2 ? b[S_WZ] : (R)1;
            for (int i = 1; i <= La; ++i) {
                R v = cA * I[(i - 1) * si];
                if (i > 1) v = fma((R)(i - 1) * b10, I[(i - 2) * si], v);
                I[i * si] = v;
            }
            for (int j = 1; j <= Lb; ++j)
                for (int i = 0; i <= La; ++i) {
                    const int e = i * si + j * sj;
                    R v = cB * I[e - sj];
                    if (j > 1) v = fma((R)(j - 1) * b10, I[e - 2 * sj], v);
                    if (i > 0) v = fma((R)i * b10, I[e - si - sj], v);
                    I[e] = v;
                }
            for (int k = 1; k <= Lc; ++k)
                for (int i = 0; i <= La; ++i)
                    for (int j = 0; j <= Lb; ++j) {
                        const int e = i * si + j * sj + k * sk;
                        R v = cC * I[e - sk];
                        if (k > 1) v = fma((R)(k - 1) * b01, I[e - 2 * sk], v);
                        if (i > 0) v = fma((R)i * b00, I[e - si - sk], v);
                        if (j > 0) v = fma((R)j * b00, I[e - sj - sk], v);
                        I[e] = v;
                    }
            for (int l = 1; l <= Ld; ++l)
                for (int k = 0; k <= Lc; ++k)
                    for (int i = 0; i <= La; ++i)
                        for (int j = 0; j <= Lb; ++j) {
                            const int e = i * si + j * sj + k * sk + l;
                            R v = cD * I[e - 1];
                            if (l > 1) v = fma((R)(l - 1) * b01, I[e - 2], v);
                            if (k > 0) v = fma((R)k * b01, I[e - sk - 1], v);
                            if (i > 0) v = fma((R)i * b00, I[e - si - 1], v);
                            if (j > 0) v = fma((R)j * b00, I[e - sj - 1], v);
                            I[e] = v;
                        }
        }
        __syncthreads();
        // D: quadrature of each (quartet, output); primitive quartets summed in FP64
        const bool last = prim + 1 == maxprim_s;
        for (int it = tid; it < qn * g.neri; it += kGenThreads) {
            const int q = it / g.neri, o = it - q * g.neri;
            int t = o;
            const int id = t % g.n[3];
            t /= g.n[3];
            const int ic = t % g.n[2];
            t /= g.n[2];
            const int ib = t % g.n[1], ia = t / g.n[1];
            int off[3];
            for (int x = 0; x < 3; ++x)
                off[x] = c_cart[La][ia][x] * si + c_cart[Lb][ib][x] * sj + c_cart[Lc][ic][x] * sk +
                         c_cart[Ld][id][x];
            const R *Ix = I_s + (size_t)(q * 3 + 0) * g.nrys * g.iblk + off[0];
            const R *Iy = I_s + (size_t)(q * 3 + 1) * g.nrys * g.iblk + off[1];
            const R *Iz = I_s + (size_t)(q * 3 + 2) * g.nrys * g.iblk + off[2];
            R s = (R)0;
            for (int mu = 0; mu < g.nrys; ++mu) s = fma(Ix[mu * g.iblk] * Iy[mu * g.iblk], Iz[mu * g.iblk], s);
            double *dst = out + (q0 + q) * (long long)g.neri + ia * args.ostride[0] + ib * args.ostride[1] +
                          ic * args.ostride[2] + id * args.ostride[3];
            const double v = (prim == 0 ? 0.0 : *dst) + RTraits<R>::to_f64(s);
            *dst = v;
            if (last && !(fabs(v) <= 1.7976931348623157e308)) atomicOr(args.err, 1);
        }
        __syncthreads();
    }
}

// eps = b_max / (2^(bits-1) - 1) of each quartet (Eq. 9), b_max from the FP64 values; one warp
// per quartet
__global__ void generic_scales_kernel(const double *__restrict__ v, long long nq, int neri, int bits,
                                      float *__restrict__ scales) {
    const long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const double *x = v + q * neri;
    double m = 0.0;
    for (int i = lane; i < neri; i += 32) m = fmax(m, fabs(x[i]));
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
    if (lane == 0) scales[q] = (float)(m / (double)((1u << (bits - 1)) - 1u));
}

// n-bit codes q = ANINT(x / eps) (Eq. 10), clamped to +-(2^(bits-1) - 1), packed LSB first: one
// thread per output word gathers the (parts of the) codes that fall in it; words past the last
// code are zero
__global__ void generic_pack_kernel(const double *__restrict__ v, long long nvals, int neri, int bits,
                                    const float *__restrict__ scales, uint32_t *__restrict__ packed,
                                    long long nwords) {
    const double M = (double)((1u << (bits - 1)) - 1u);
    const uint32_t mask = (1u << bits) - 1u;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < nwords;
         w += (long long)gridDim.x * blockDim.x) {
        const long long b0 = w * 32;
        const long long first = b0 / bits, lastc = (b0 + 31) / bits;
        uint32_t word = 0u;
        for (long long c = first; c <= lastc && c < nvals; ++c) {
            const float eps = scales[c / neri];
            const double inv = eps > 0.0f ? 1.0 / (double)eps : 0.0;
            double r = round(v[c] * inv);
            r = r > M ? M : (r < -M ? -M : r);
            const uint32_t code = (uint32_t)(int)r & mask;
            const long long s = c * bits - b0;
            word |= s >= 0 ? code << s : code >> (-s);
        }
        packed[w] = word;
    }
}

template <typename R>
cudaError_t run_values(const ShellsDev &sh, const Tables &tb, const ClassArgs &a, const GenShape &g,
                       double *out, cudaStream_t stream) {
    auto kern = eri_generic_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (a.nq + g.q - 1) / g.q;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)tiles, kGenThreads, g.smem, stream>>>(sh, tb, a, g, out);
    return cudaGetLastError();
}

// quartets per compressed chunk: a multiple of 32 (every chunk starts on a packed word)
long long chunk_quartets(int neri, size_t scratch_bytes) {
    long long c = (long long)(scratch_bytes / (sizeof(double) * (size_t)neri)) / 32 * 32;
    return c;
}

}  // namespace

cudaError_t launch_generic(const ShellsDev &sh, const Tables &tb, const ClassArgs &a, const int L[4],
                           bool mixed, double *scratch, size_t scratch_bytes, cudaStream_t stream) {
    if (a.nq <= 0) return cudaSuccess;
    const GenShape g = mixed ? gen_shape<float>(L) : gen_shape<double>(L);
    if (g.smem > 227 * 1024) return cudaErrorInvalidValue;
    if (a.out_fp64)
        return mixed ? run_values<float>(sh, tb, a, g, a.out_fp64, stream)
                     : run_values<double>(sh, tb, a, g, a.out_fp64, stream);
    const long long chunk = chunk_quartets(g.neri, scratch_bytes);
    if (chunk < 32 || !scratch) return cudaErrorInvalidValue;
    for (long long c0 = 0; c0 < a.nq; c0 += chunk) {
        ClassArgs ac = a;
        ac.quartets = a.quartets + c0;
        ac.nq = std::min(chunk, a.nq - c0);
        cudaError_t e = mixed ? run_values<float>(sh, tb, ac, g, scratch, stream)
                              : run_values<double>(sh, tb, ac, g, scratch, stream);
        if (e != cudaSuccess) return e;
        generic_scales_kernel<<<(unsigned)((ac.nq * 32 + 255) / 256), 256, 0, stream>>>(
            scratch, ac.nq, g.neri, a.bits, a.scales + c0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const long long w0 = c0 * g.neri * a.bits / 32;
        const long long nw = (c0 + ac.nq == a.nq) ? a.seg_words - w0 : ac.nq * g.neri * a.bits / 32;
        const long long blocks = std::min<long long>((nw + 255) / 256, 152LL * 16);
        generic_pack_kernel<<<(unsigned)std::max<long long>(1, blocks), 256, 0, stream>>>(
            scratch, ac.nq * g.neri, g.neri, a.bits, a.scales + c0, a.packed + w0, nw);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int generic_launches(long long nq, int neri, bool compressed, size_t scratch_bytes) {
    if (nq <= 0) return 0;
    if (!compressed) return 1;
    const long long chunk = chunk_quartets(neri, scratch_bytes);
    return chunk > 0 ? 3 * (int)((nq + chunk - 1) / chunk) : 0;
}

const char *generic_kernel_names(bool mixed, bool compressed) {
    if (compressed)
        return mixed ? "eri_generic_kernel<float> + generic_scales_kernel + generic_pack_kernel"
                     : "eri_generic_kernel<double> + generic_scales_kernel + generic_pack_kernel";
    return mixed ? "eri_generic_kernel<float>" : "eri_generic_kernel<double>";
}

}  // namespace eri
