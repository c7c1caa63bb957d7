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
#include <vector>

#include "eri_internal.h"
#include "eri_kernels.cuh"

namespace eri {

namespace {

constexpr int kGenThreads = 256;
constexpr int kGenAcc = 8;  // outputs per thread summed over primitives in registers
// B, C values per (quartet, root): the slots of phase_setup plus C00 relative to B and C00'
// relative to D
constexpr int kGenCB = S_N, kGenCD = S_N + 3, kGenSN = S_N + 6;
constexpr int kGenSNP = kGenSN + 1;  // odd stride of the (quartet, root) records: distinct banks

// geometry without the choice of transfer direction (the four-index recursion needs none)
struct GenGeo {
    static constexpr bool SWAB_OK = false, SWCD_OK = false;
};

struct GenShape {
    int L[4];        // canonical angular momenta
    int n[4];        // Cartesian components per shell
    int nrys, neri;  // roots, ERIs per quartet
    int iblk;        // 2-D integrals per (root, axis): (La+1)(Lb+1)(Lc+1)(Ld+1)
    int iblkp;       // their stride in shared memory, odd so that the blocks the threads of a
                     // warp build start in distinct banks
    int q;           // quartets per CTA
    int bc_off, i_off, smem;  // dynamic shared memory layout (bytes)
};

template <typename R>
GenShape gen_shape(const int L[4], int qmax = 64) {
    GenShape g{};
    for (int k = 0; k < 4; ++k) {
        g.L[k] = L[k];
        g.n[k] = ncart(L[k]);
    }
    g.nrys = (L[0] + L[1] + L[2] + L[3]) / 2 + 1;
    g.neri = g.n[0] * g.n[1] * g.n[2] * g.n[3];
    g.iblk = (L[0] + 1) * (L[1] + 1) * (L[2] + 1) * (L[3] + 1);
    g.iblkp = g.iblk | 1;
    const int geo = G_N * 8, bc = g.nrys * kGenSNP * (int)sizeof(R), ib = 3 * g.nrys * g.iblkp * (int)sizeof(R);
    const int perq = geo + bc + ib + 16;
    // quartets per CTA: within the shared-memory budget, and (for classes of at most
    // kGenThreads * kGenAcc outputs) few enough that the primitive sums stay in registers
    g.q = std::max(1, std::min(qmax, (96 * 1024) / perq));
    if (g.neri <= kGenThreads * kGenAcc) g.q = std::max(1, std::min(g.q, kGenThreads * kGenAcc / g.neri));
    g.bc_off = g.q * geo;
    g.i_off = ((g.bc_off + g.q * bc + 15) / 16) * 16;
    g.smem = g.i_off + g.q * ib;
    return g;
}

// One tile: quartets [q0, q0 + qn) of the class of `args`, ERIs summed over primitive quartets
// in FP64 into out[q * n_ERIQ + generic index], q = 0..qn-1 (out = the tile's first quartet).
// Every thread of the CTA calls it; it begins and ends with a barrier.
template <typename R>
__device__ __forceinline__ void generic_tile(const ShellsDev &sh, const Tables &tb, const ClassArgs &args,
                                             const GenShape &g, long long q0, int qn, double *__restrict__ out,
                                             unsigned char *smem, int &maxprim_s) {
    double *geo_s = reinterpret_cast<double *>(smem);
    R *bc_s = reinterpret_cast<R *>(smem + g.bc_off);
    R *I_s = reinterpret_cast<R *>(smem + g.i_off);
    const int tid = threadIdx.x;
    const int La = g.L[0], Lb = g.L[1], Lc = g.L[2], Ld = g.L[3];
    // strides of I(i, j, k, l) within one (root, axis) block
    const int sk = Ld + 1, sj = (Lc + 1) * sk, si = (Lb + 1) * sj;
    const bool in_regs = qn * g.neri <= kGenThreads * kGenAcc;
    double acc[kGenAcc];
#pragma unroll
    for (int k = 0; k < kGenAcc; ++k) acc[k] = 0.0;
    __syncthreads();
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
            R *b = bc_s + (size_t)it * kGenSNP;
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
            const R *b = bc_s + (size_t)(q * g.nrys + mu) * kGenSNP;
            R *I = I_s + (size_t)it * g.iblkp;  // block (q, mu, xi): consecutive threads, odd stride
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
        // D: quadrature of each (quartet, output); primitive quartets summed in FP64, in the
        // thread's registers when the tile has at most kGenAcc outputs per thread (the same
        // outputs every primitive), else in `out`
        const bool last = prim + 1 == maxprim_s;
        auto quad = [&](int it, double *&dst) -> R {
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
            const R *I0 = I_s + (size_t)q * g.nrys * 3 * g.iblkp;
            const R *Ix = I0 + off[0], *Iy = I0 + g.iblkp + off[1], *Iz = I0 + 2 * g.iblkp + off[2];
            const int ms = 3 * g.iblkp;  // next root
            R s = (R)0;
            for (int mu = 0; mu < g.nrys; ++mu) s = fma(Ix[mu * ms] * Iy[mu * ms], Iz[mu * ms], s);
            dst = out + q * (long long)g.neri + ia * args.ostride[0] + ib * args.ostride[1] + ic * args.ostride[2] +
                  id * args.ostride[3];
            return s;
        };
        if (in_regs) {
#pragma unroll
            for (int k = 0; k < kGenAcc; ++k) {
                const int it = tid + k * kGenThreads;
                if (it < qn * g.neri) {
                    double *dst;
                    acc[k] += RTraits<R>::to_f64(quad(it, dst));
                    if (last) {
                        *dst = acc[k];
                        if (!(fabs(acc[k]) <= 1.7976931348623157e308)) atomicOr(args.err, 1);
                    }
                }
            }
        } else {
            for (int it = tid; it < qn * g.neri; it += kGenThreads) {
                double *dst;
                const R s = quad(it, dst);
                const double v = (prim == 0 ? 0.0 : *dst) + RTraits<R>::to_f64(s);
                *dst = v;
                if (last && !(fabs(v) <= 1.7976931348623157e308)) atomicOr(args.err, 1);
            }
        }
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(kGenThreads)
eri_generic_kernel(ShellsDev sh, Tables tb, ClassArgs args, GenShape g, double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int maxprim_s;
    const long long q0 = (long long)blockIdx.x * g.q;
    const int qn = (int)((args.nq - q0) < g.q ? (args.nq - q0) : g.q);
    generic_tile<R>(sh, tb, args, g, q0, qn, out + q0 * (long long)g.neri, smem, maxprim_s);
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

// ---------------------------------------------------------------------------------------------
// One persistent launch for every class of a plan: a work queue of tiles (class, quartets
// [q0, q0 + q)) over all classes, pulled by the resident CTAs from one atomic counter, so
// quartets of uneven class and contraction degree balance across the GPU.  Each tile's FP64
// values go to the CTA's slot of a scratch buffer and are compressed in the same launch: b_max
// and eps per quartet (Eq. 9), then the codes (Eq. 10) packed one output word per thread; words
// that a tile shares with its neighbour tile are OR-ed in (the output is zeroed before the
// launch), the others stored.

struct QueueClass {
    ClassArgs a;           // quartets, permutation, output strides, packed segment and scales
    GenShape g;            // shape and shared-memory layout (common quartet cap)
    long long first_tile;  // first tile of the class in the queue
};

constexpr int kQueueQmax = 128;

template <typename R>
__global__ void __launch_bounds__(kGenThreads)
eri_queue_kernel(ShellsDev sh, Tables tb, const QueueClass *__restrict__ classes, int n_classes,
                 long long n_tiles, unsigned long long *counter, double *__restrict__ scratch,
                 long long slot_doubles, int bits, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int maxprim_s;
    __shared__ long long item_s;
    __shared__ int cls_s;
    __shared__ unsigned long long bmax_s[kQueueQmax];
    __shared__ float eps_s[kQueueQmax];
    const int tid = threadIdx.x;
    double *vals = scratch + (long long)blockIdx.x * slot_doubles;
    const double M = (double)((1u << (bits - 1)) - 1u);
    const uint32_t mask = (1u << bits) - 1u;
    for (;;) {
        if (tid == 0) {
            item_s = (long long)atomicAdd(counter, 1ull);
            int lo = 0, hi = n_classes - 1;  // last class whose first tile <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (classes[mid].first_tile <= item_s) lo = mid; else hi = mid - 1;
            }
            cls_s = lo;
        }
        __syncthreads();
        const long long item = item_s;
        if (item >= n_tiles) break;
        const QueueClass &qc = classes[cls_s];
        const ClassArgs a = qc.a;
        const GenShape g = qc.g;
        const long long q0 = (item - qc.first_tile) * g.q;
        const int qn = (int)((a.nq - q0) < g.q ? (a.nq - q0) : g.q);
        generic_tile<R>(sh, tb, a, g, q0, qn, vals, smem, maxprim_s);
        // b_max per quartet (non-negative IEEE values order like their bit patterns)
        for (int q = tid; q < qn; q += kGenThreads) bmax_s[q] = 0ull;
        __syncthreads();
        for (int it = tid; it < qn * g.neri; it += kGenThreads) {
            const double v = fabs(vals[it]);
            if (!(v <= 1.7976931348623157e308)) atomicOr(err, 1);
            atomicMax(bmax_s + it / g.neri, (unsigned long long)__double_as_longlong(v));
        }
        __syncthreads();
        for (int q = tid; q < qn; q += kGenThreads) {
            const float e = (float)(__longlong_as_double((long long)bmax_s[q]) / M);
            eps_s[q] = e;
            a.scales[q0 + q] = e;
        }
        __syncthreads();
        // codes of the tile's values [c0, c1) at stream bits [c0 * bits, c1 * bits)
        const long long c0 = q0 * g.neri, c1 = (q0 + qn) * (long long)g.neri;
        const long long b0 = c0 * bits, b1 = c1 * bits;
        for (long long w = (b0 >> 5) + tid; w < ((b1 + 31) >> 5); w += kGenThreads) {
            const long long wb = w * 32;
            long long first = wb / bits, last = (wb + 31) / bits;
            first = first < c0 ? c0 : first;
            last = last >= c1 ? c1 - 1 : last;
            uint32_t word = 0u;
            for (long long c = first; c <= last; ++c) {
                const float e = eps_s[(c - c0) / g.neri];
                const double inv = e > 0.0f ? 1.0 / (double)e : 0.0;
                double r = round(vals[c - c0] * inv);
                r = r > M ? M : (r < -M ? -M : r);
                const uint32_t code = (uint32_t)(int)r & mask;
                const long long sh_ = c * bits - wb;
                word |= sh_ >= 0 ? code << sh_ : code >> (-sh_);
            }
            if (wb >= b0 && wb + 32 <= b1)
                a.packed[w] = word;
            else
                atomicOr(a.packed + w, word);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_queue(const ShellsDev &sh, const Tables &tb, const QueueSpec *classes, int n_classes,
                         bool mixed, int bits, int *err, void *d_table, unsigned long long *d_counter,
                         double *scratch, size_t scratch_bytes, int device, cudaStream_t stream) {
    if (n_classes <= 0) return cudaSuccess;
    std::vector<QueueClass> qc(n_classes);
    long long tiles = 0;
    int smem = 0;
    long long slot = 1;
    for (int i = 0; i < n_classes; ++i) {
        qc[i].a = classes[i].a;
        qc[i].g = mixed ? gen_shape<float>(classes[i].L, kQueueQmax) : gen_shape<double>(classes[i].L, kQueueQmax);
        qc[i].first_tile = tiles;
        tiles += (classes[i].a.nq + qc[i].g.q - 1) / qc[i].g.q;
        smem = std::max(smem, qc[i].g.smem);
        slot = std::max(slot, (long long)qc[i].g.q * qc[i].g.neri);
    }
    if (smem > 227 * 1024 - 2048) return cudaErrorInvalidValue;
    void (*kern)(ShellsDev, Tables, const QueueClass *, int, long long, unsigned long long *, double *,
                 long long, int, int *) = mixed ? eri_queue_kernel<float> : eri_queue_kernel<double>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGenThreads, smem)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return e;
    long long grid = std::min<long long>(tiles, (long long)std::max(1, per_sm) * sms);
    grid = std::min<long long>(grid, (long long)(scratch_bytes / (sizeof(double) * (size_t)slot)));
    if (grid < 1) return cudaErrorInvalidValue;
    if ((size_t)n_classes * sizeof(QueueClass) > queue_table_bytes()) return cudaErrorInvalidValue;
    e = cudaMemcpyAsync(d_table, qc.data(), (size_t)n_classes * sizeof(QueueClass), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kGenThreads, smem, stream>>>(sh, tb, static_cast<const QueueClass *>(d_table), n_classes,
                                                        tiles, d_counter, scratch, slot, bits, err);
    return cudaGetLastError();
}

size_t queue_table_bytes() { return (size_t)kNumClassIds * sizeof(QueueClass); }

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
