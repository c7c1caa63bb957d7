// eri_digest.cu -- consumer side of the compressed ERIs: decompression (Sec. II-D, Eq. 11)
// fused with their contraction against a density matrix into the Coulomb and exchange
// matrices,
//   J[mu, nu]  += (mu nu | lam sig) D[lam, sig],     K[mu, lam] += (mu nu | lam sig) D[nu, sig],
// the use Sec. I and Sec. II-D give for computing and storing ERIs compressed (the matrices
// an SCF or AIMD step rebuilds from the stored integrals).
//
// A quartet's block e[a][b][c][d] (codes q times the quartet's eps) contributes through each of
// the eight index permutations of Sec. II-B that give a distinct ordered shell quartet
// (permutations that map the quartet onto itself are counted once).  For the eight
// permutations the twelve contractions needed fall into six "index-pair passes": a pass fixes
// two positions (x, y) of the block and sums over the other two (u, w) against the D block
// D[u, w] and its transpose D[w, u]:
//   pass (a,b): T1 = sum e D[c,d] -> J[a,b] (perm 1), J[b,a] (perm 2);
//               T2 = sum e D[d,c] -> J[a,b] (perm 3), J[b,a] (perm 4)
//   pass (c,d): T3 = sum e D[a,b] -> J[c,d] (5), J[d,c] (6); T4 = sum e D[b,a] -> J[c,d] (7), J[d,c] (8)
//   pass (a,c): sum e D[b,d] -> K[a,c] (1);  sum e D[d,b] -> K[c,a] (5)
//   pass (b,c): sum e D[a,d] -> K[b,c] (2);  sum e D[d,a] -> K[c,b] (7)
//   pass (a,d): sum e D[b,c] -> K[a,d] (3);  sum e D[c,b] -> K[d,a] (6)
//   pass (b,d): sum e D[a,c] -> K[b,d] (4);  sum e D[c,a] -> K[d,b] (8)
// with the permutations 1..8 = (abcd), (bacd), (abdc), (badc), (cdab), (dcab), (cdba), (dcba).
//
// GPU mapping: one CTA per tile of quartets of one class.  The tile's codes are decoded into
// shared memory as FP32 integers (exact for widths <= 24), the twelve D blocks between the
// quartet's four shells are staged in FP32, and each thread takes (quartet, pass, x, y) items,
// forms both sums in FP32, scales them by eps and adds them to J and K in FP64 (device
// atomics, so the summation order of the FP64 accumulation varies between runs).
#include <algorithm>
#include <vector>

#include "eri_internal.h"

namespace eri {

namespace {

constexpr int kDigestThreads = 256;
// dynamic shared memory of a tile: 47 KB, so that with the kernel's static shared memory (the
// class parameters) a CTA stays within the 48 KB available without an opt-in
constexpr int kDigestSmem = 47 * 1024;

// the twelve D blocks (x, y), x != y, in x-major order
__constant__ int c_bx[12] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3};
__constant__ int c_by[12] = {1, 2, 3, 0, 2, 3, 0, 1, 3, 0, 1, 2};
// pass p fixes positions (PX, PY) and sums over (PU, PW)
__constant__ int c_px[6] = {0, 2, 0, 1, 0, 1};
__constant__ int c_py[6] = {1, 3, 2, 2, 3, 3};
__constant__ int c_pu[6] = {2, 0, 1, 0, 1, 0};
__constant__ int c_pw[6] = {3, 1, 3, 3, 2, 2};

struct DigestArgs {
    const int4 *quartets;  // class-sorted shell ids of the class
    long long nq;
    const uint32_t *packed;  // class segment of the packed stream
    const float *scales;     // eps of the class's quartets
    const int *bfoff;        // first basis function of every shell
    const float *D;          // density matrix, FP32, row major
    long long nbf;
    double *J, *K;
    int bits;
    int unique8;
    int n[4];      // Cartesian components of the four positions
    int st[4];     // strides of the four positions in the quartet's block
    int neri;
    int T;         // quartets per tile
    int nD;        // staged D values per quartet
    int boff[16];  // offset of D block (x, y) (index x*4 + y) in a quartet's D area
    int rstart[13];  // first row of each of the 12 blocks (x != y, in x-major order); [12] = rows
    int NI;        // items per quartet
    int ioff[7];   // first item of each pass
};

// Which of the eight permutations give a distinct ordered shell quartet (bit p-1 for
// permutation p): a permutation equal, as a tuple of shell ids, to an earlier one is dropped.
__device__ __forceinline__ int perm_mask(int4 s, bool unique8) {
    if (!unique8) return 1;
    const int t[8][4] = {{s.x, s.y, s.z, s.w}, {s.y, s.x, s.z, s.w}, {s.x, s.y, s.w, s.z},
                         {s.y, s.x, s.w, s.z}, {s.z, s.w, s.x, s.y}, {s.w, s.z, s.x, s.y},
                         {s.z, s.w, s.y, s.x}, {s.w, s.z, s.y, s.x}};
    int mask = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        bool fresh = true;
#pragma unroll
        for (int r = 0; r < p; ++r)
            fresh &= !(t[p][0] == t[r][0] && t[p][1] == t[r][1] && t[p][2] == t[r][2] &&
                       t[p][3] == t[r][3]);
        mask |= fresh ? (1 << p) : 0;
    }
    return mask;
}

// Coefficients (0 or 1) of the two sums of pass p in its two destinations:
// dest 1 = M[x, y] gets c[0] S + c[1] S', dest 2 = M[y, x] gets c[2] S + c[3] S'.
__device__ __forceinline__ void pass_coefs(int p, int m, int c[4]) {
    auto b = [m](int perm) { return (m >> (perm - 1)) & 1; };
    switch (p) {
        case 0: c[0] = b(1); c[1] = b(3); c[2] = b(2); c[3] = b(4); break;
        case 1: c[0] = b(5); c[1] = b(7); c[2] = b(6); c[3] = b(8); break;
        case 2: c[0] = b(1); c[1] = 0; c[2] = 0; c[3] = b(5); break;
        case 3: c[0] = b(2); c[1] = 0; c[2] = 0; c[3] = b(7); break;
        case 4: c[0] = b(3); c[1] = 0; c[2] = 0; c[3] = b(6); break;
        default: c[0] = b(4); c[1] = 0; c[2] = 0; c[3] = b(8); break;
    }
}

// SYM: the caller's D is symmetric.  Then S = S' in every pass (D[u][w] = D[w][u]) and the two
// destinations M[x][y], M[y][x] of an item receive equal totals over the whole sum, so each item
// forms one sum and adds all of its coefficient to M[x][y] alone; the finished matrices are
// symmetrised afterwards, M = (M + M^T) / 2 (symmetrise_kernel), which restores every entry.
//
// One launch covers every class: CTA b takes tile b - tile_start[c] of the class c with
// tile_start[c] <= b < tile_start[c + 1] (the classes' parameters in `args`, copied to shared
// memory by the CTA), so small classes do not leave the GPU idle between launches.
template <bool SYM>
__global__ void __launch_bounds__(kDigestThreads)
digest_kernel(const DigestArgs *__restrict__ args, const long long *__restrict__ tile_start, int n_classes) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DigestArgs A;
    __shared__ long long tile_s;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_classes - 1;  // last class with tile_start <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (tile_start[mid] <= (long long)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        tile_s = ((long long)blockIdx.x - tile_start[lo]) | ((long long)lo << 40);
    }
    __syncthreads();
    {
        const int c = (int)(tile_s >> 40);
        const int *src = reinterpret_cast<const int *>(args + c);
        int *dst = reinterpret_cast<int *>(&A);
        for (int i = threadIdx.x; i < (int)(sizeof(DigestArgs) / 4); i += kDigestThreads) dst[i] = src[i];
    }
    __syncthreads();
    int *meta = reinterpret_cast<int *>(smem);               // T x 8: bf offsets, mask, eps
    float *e_s = reinterpret_cast<float *>(meta + A.T * 8);  // T x neri codes
    float *d_s = e_s + (size_t)A.T * A.neri;                 // T x nD D values
    const long long q0 = (tile_s & ((1LL << 40) - 1)) * A.T;
    const int tn = (int)((A.nq - q0) < A.T ? (A.nq - q0) : A.T);
    const int tid = threadIdx.x;

    for (int t = tid; t < tn; t += kDigestThreads) {
        const int4 s = A.quartets[q0 + t];
        int *m = meta + t * 8;
        m[0] = A.bfoff[s.x];
        m[1] = A.bfoff[s.y];
        m[2] = A.bfoff[s.z];
        m[3] = A.bfoff[s.w];
        m[4] = perm_mask(s, A.unique8 != 0);
        m[5] = __float_as_int(A.scales[q0 + t]);
    }
    // codes of the tile: fields q0*neri .. (q0+tn)*neri of the class's stream (Eq. 11 without
    // the scale, which is applied once per sum)
    const int nv = tn * A.neri;
    const long long f0 = q0 * A.neri;
    const uint32_t fmask = (1u << A.bits) - 1u;
    for (int v = tid; v < nv; v += kDigestThreads) {
        const unsigned long long bit = (unsigned long long)(f0 + v) * (unsigned)A.bits;
        const long long w = (long long)(bit >> 5);
        const int off = (int)(bit & 31);
        uint32_t raw = __ldg(A.packed + w) >> off;
        if (off + A.bits > 32) raw |= __ldg(A.packed + w + 1) << (32 - off);
        raw &= fmask;
        const int code = (int)(raw << (32 - A.bits)) >> (32 - A.bits);  // sign extension
        e_s[v] = (float)code;
    }
    __syncthreads();
    // the D blocks between the quartet's shells, D[o_x + i][o_y + j] for x != y: one thread per
    // (quartet, block row), whose at most 10 loads are independent
    const int rows = A.rstart[12];
    for (int idx = tid; idx < tn * rows; idx += kDigestThreads) {
        const int t = idx / rows;
        const int r = idx - t * rows;
        int b = 0;
#pragma unroll
        for (int k = 1; k < 12; ++k) b += r >= A.rstart[k];
        const int x = c_bx[b], y = c_by[b];
        const int i = r - A.rstart[b], ny = A.n[y];
        const int *m = meta + t * 8;
        const float *src = A.D + (long long)(m[x] + i) * A.nbf + m[y];
        float *dst = d_s + t * A.nD + A.boff[x * 4 + y] + i * ny;
#pragma unroll 10
        for (int j = 0; j < ny; ++j) dst[j] = __ldg(src + j);
    }
    __syncthreads();
    for (int it = tid; it < tn * A.NI; it += kDigestThreads) {
        const int t = it / A.NI;
        const int r = it - t * A.NI;
        int p = 0;
#pragma unroll
        for (int k = 1; k < 6; ++k) p += r >= A.ioff[k];
        const int *m = meta + t * 8;
        int c[4];
        pass_coefs(p, m[4], c);
        if ((c[0] | c[1] | c[2] | c[3]) == 0) continue;
        const int x = c_px[p], y = c_py[p], u = c_pu[p], w = c_pw[p];
        const int loc = r - A.ioff[p];
        const int ix = loc / A.n[y], iy = loc - (loc / A.n[y]) * A.n[y];
        const int nu = A.n[u], nw = A.n[w], su = A.st[u], sw = A.st[w];
        const float *ep = e_s + t * A.neri + ix * A.st[x] + iy * A.st[y];
        const float *d1 = d_s + t * A.nD + A.boff[u * 4 + w];  // D[u][w], row length nw
        const float *d2 = d_s + t * A.nD + A.boff[w * 4 + u];  // D[w][u], row length nu
        const float eps = __int_as_float(m[5]);
        double *M = p < 2 ? A.J : A.K;
        const long long row = m[x] + ix, col = m[y] + iy;
        if constexpr (SYM) {
            float S = 0.0f;
#pragma unroll 1
            for (int iu = 0; iu < nu; ++iu)
#pragma unroll 2
                for (int iw = 0; iw < nw; ++iw) S = fmaf(ep[iu * su + iw * sw], d1[iu * nw + iw], S);
            const float k = (float)(c[0] + c[1] + c[2] + c[3]);
            atomicAdd(M + row * A.nbf + col, f32_to_f64(S * (k * eps)));
        } else {
            float S = 0.0f, S2 = 0.0f;
#pragma unroll 1
            for (int iu = 0; iu < nu; ++iu)
#pragma unroll 2
                for (int iw = 0; iw < nw; ++iw) {
                    const float e = ep[iu * su + iw * sw];
                    S = fmaf(e, d1[iu * nw + iw], S);
                    S2 = fmaf(e, d2[iw * nu + iu], S2);
                }
            const float v1 = (c[0] ? S : 0.0f) + (c[1] ? S2 : 0.0f);
            const float v2 = (c[2] ? S : 0.0f) + (c[3] ? S2 : 0.0f);
            if (c[0] | c[1]) atomicAdd(M + row * A.nbf + col, f32_to_f64(v1 * eps));
            if (c[2] | c[3]) atomicAdd(M + col * A.nbf + row, f32_to_f64(v2 * eps));
        }
    }
}

// M = (M + M^T) / 2 for an n x n row-major matrix, one thread per pair i < j.
__global__ void symmetrise_kernel(double *__restrict__ M, long long n) {
    const long long pairs = n * (n - 1) / 2;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < pairs;
         t += (long long)gridDim.x * blockDim.x) {
        long long i = (long long)((sqrt(8.0 * (double)t + 1.0) + 1.0) * 0.5);  // row, i >= 1
        while (i * (i - 1) / 2 > t) --i;
        while ((i + 1) * i / 2 <= t) ++i;
        const long long j = t - i * (i - 1) / 2;  // 0 <= j < i
        const double v = 0.5 * (M[i * n + j] + M[j * n + i]);
        M[i * n + j] = v;
        M[j * n + i] = v;
    }
}

__global__ void density_to_f32_kernel(const double *__restrict__ D, long long n, float *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = f64_to_f32(D[i]);
}

int ncart_d(int L) { return (L + 1) * (L + 2) / 2; }

}  // namespace

cudaError_t digest_density_f32(const double *D, long long n, float *out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    density_to_f32_kernel<<<(unsigned)blocks, 256, 0, stream>>>(D, n, out);
    return cudaGetLastError();
}

cudaError_t digest_symmetrise(double *M, long long n, cudaStream_t stream) {
    if (n < 2) return cudaSuccess;
    const long long pairs = n * (n - 1) / 2;
    long long blocks = (pairs + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    symmetrise_kernel<<<(unsigned)blocks, 256, 0, stream>>>(M, n);
    return cudaGetLastError();
}

size_t digest_table_bytes() { return 256 * sizeof(DigestArgs) + 257 * sizeof(long long); }

cudaError_t digest_all(const DigestClass *classes, int n_classes, int bits, bool unique8, bool symmetric,
                       const int *bfoff, const float *D32, long long nbf, double *J, double *K,
                       void *d_table, cudaStream_t stream) {
    if (n_classes <= 0) return cudaSuccess;
    if (n_classes > 256) return cudaErrorInvalidValue;
    std::vector<DigestArgs> args(n_classes);
    std::vector<long long> start(n_classes + 1);
    size_t smem_max = 0;
    long long tiles = 0;
    for (int k = 0; k < n_classes; ++k) {
        const DigestClass &c = classes[k];
        DigestArgs &A = args[k];
        A = DigestArgs{};
        A.quartets = c.quartets;
        A.nq = c.nq;
        A.packed = c.packed;
        A.scales = c.scales;
        A.bfoff = bfoff;
        A.D = D32;
        A.nbf = nbf;
        A.J = J;
        A.K = K;
        A.bits = bits;
        A.unique8 = unique8 ? 1 : 0;
        const int L[4] = {(c.cls >> 6) & 3, (c.cls >> 4) & 3, (c.cls >> 2) & 3, c.cls & 3};
        for (int x = 0; x < 4; ++x) A.n[x] = ncart_d(L[x]);
        A.st[3] = 1;
        for (int x = 2; x >= 0; --x) A.st[x] = A.st[x + 1] * A.n[x + 1];
        A.neri = A.st[0] * A.n[0];
        int o = 0;
        for (int b = 0; b < 16; ++b) {
            const int x = b >> 2, y = b & 3;
            A.boff[b] = o;
            if (x != y) o += A.n[x] * A.n[y];
        }
        A.nD = o;
        const int bx[12] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3};
        A.rstart[0] = 0;
        for (int b = 0; b < 12; ++b) A.rstart[b + 1] = A.rstart[b] + A.n[bx[b]];
        const int px[6] = {0, 2, 0, 1, 0, 1}, py[6] = {1, 3, 2, 2, 3, 3};
        A.ioff[0] = 0;
        for (int p = 0; p < 6; ++p) A.ioff[p + 1] = A.ioff[p] + A.n[px[p]] * A.n[py[p]];
        A.NI = A.ioff[6];
        const int perq = 4 * (8 + A.neri + A.nD);
        int T = kDigestSmem / perq;
        T = T < 1 ? 1 : (T > 128 ? 128 : T);
        A.T = T;
        if ((size_t)T * perq > (size_t)kDigestSmem) return cudaErrorInvalidValue;
        smem_max = std::max(smem_max, (size_t)T * perq);
        start[k] = tiles;
        tiles += (c.nq + T - 1) / T;
    }
    start[n_classes] = tiles;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    DigestArgs *d_args = static_cast<DigestArgs *>(d_table);
    long long *d_start = reinterpret_cast<long long *>(static_cast<char *>(d_table) + 256 * sizeof(DigestArgs));
    cudaError_t e = cudaMemcpyAsync(d_args, args.data(), n_classes * sizeof(DigestArgs), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_start, start.data(), (n_classes + 1) * sizeof(long long), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return e;
    if (symmetric)
        digest_kernel<true><<<(unsigned)tiles, kDigestThreads, smem_max, stream>>>(d_args, d_start, n_classes);
    else
        digest_kernel<false><<<(unsigned)tiles, kDigestThreads, smem_max, stream>>>(d_args, d_start, n_classes);
    return cudaGetLastError();
}

}  // namespace eri
