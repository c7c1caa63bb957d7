// The paper's output chunks (Sec. III-C, compress-store loops): every quartet's n-bit codes
// are written as 512-bit words of F = floor(512/n) fields; the fields that do not fit in one
// chunk open the next, the last chunk of a quartet is zero-padded, so a quartet takes
// n_CS = ceil(n_eri / F) chunks of 64 bytes and no chunk mixes quartets.  Field j of a chunk
// holds chunk bits [j*n, j*n + n), chunk bit s being bit s%32 of the chunk's 32-bit word s/32.
//
// The compressing kernels write the dense stream (every field right after the previous one);
// this file re-lays a class's dense stream into chunks.  It is integer-only, HBM-bound work:
// one thread per output word gathers the (at most 32/n + 2) fields that overlap it from one
// or two dense words each, so reads and writes are both coalesced along the chunk.
#include <cstdint>

#include <cuda_runtime.h>

#include "eri.h"

namespace eri {
namespace {

constexpr int kChunkWords = 16;  // 512 bits

// Quartets [q0, q0 + nq) of one class.  `src` is the class's dense stream (word 0 holds stream
// bit 0), `dst` the chunk words of quartet q0.  nq * n_cs * 16 < 2^31 (host-checked), and every
// in-quartet bit offset fits 32 bits (n_eri * bits <= 50625 * 24, [gg|gg] at 24 bits).
__global__ void __launch_bounds__(256) paper512_kernel(const uint32_t *__restrict__ src,
                                                       unsigned long long q0, unsigned nq,
                                                       unsigned n_eri, unsigned n_cs, unsigned bits,
                                                       uint32_t *__restrict__ dst) {
    const unsigned F = 512u / bits;
    const unsigned total = nq * n_cs * kChunkWords;
    const uint32_t mask = (1u << bits) - 1u;  // bits <= 24
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned ch = t / kChunkWords, k = t % kChunkWords;
        const unsigned i = ch / n_cs, c = ch - i * n_cs;
        // first stream bit of this quartet's codes
        const unsigned long long qbit = (q0 + i) * (unsigned long long)n_eri * bits;
        const uint32_t *qs = src + (qbit >> 5);
        const unsigned off = (unsigned)qbit & 31u;
        const unsigned lo = 32u * k;          // chunk bits [lo, lo + 32) make this word
        const unsigned nf = min(F, n_eri - c * F);  // fields in this chunk (>= 1 since c < n_cs)
        const unsigned j0 = lo / bits;
        const unsigned j1 = min((lo + 31u) / bits, nf - 1u);
        uint32_t out = 0;
        for (unsigned j = j0; j <= j1; ++j) {
            const unsigned b = off + (c * F + j) * bits;  // field's bit within the quartet's words
            const unsigned w = b >> 5, s = b & 31u;
            uint32_t v = qs[w] >> s;
            if (s + bits > 32u) v |= qs[w + 1] << (32u - s);  // the field spills into the next word
            v &= mask;
            const int o = (int)(j * bits) - (int)lo;
            out |= o >= 0 ? v << o : v >> (-o);
        }
        dst[t] = out;
    }
}

// The same with one thread per quarter chunk (four consecutive output words, one 16-byte store):
// the quartet and chunk indices are found once per four words, and the field indices lo / bits
// and (lo + 31) / bits by a multiply with ceil(2^16 / bits) (exact for lo < 2^9 and bits <= 24:
// the product overshoots lo / bits by less than lo / 2^16 < 1 / bits).  dst 16-byte aligned.
__global__ void __launch_bounds__(256) paper512_kernel4(const uint32_t *__restrict__ src,
                                                        unsigned long long q0, unsigned nq,
                                                        unsigned n_eri, unsigned n_cs, unsigned bits,
                                                        uint4 *__restrict__ dst) {
    const unsigned F = 512u / bits;
    const unsigned inv = (65536u + bits - 1u) / bits;
    const unsigned total = nq * n_cs * (kChunkWords / 4);
    const uint32_t mask = (1u << bits) - 1u;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned ch = t >> 2, k0 = (t & 3u) * 4u;
        const unsigned i = ch / n_cs, c = ch - i * n_cs;
        const unsigned long long qbit = (q0 + i) * (unsigned long long)n_eri * bits;
        const uint32_t *qs = src + (qbit >> 5);
        const unsigned off = (unsigned)qbit & 31u;
        const unsigned nf = min(F, n_eri - c * F);
        uint32_t out[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const unsigned lo = 32u * (k0 + kk);
            const unsigned j0 = (lo * inv) >> 16;
            uint32_t o = 0;
            if (j0 < nf) {
                const unsigned j1 = min(((lo + 31u) * inv) >> 16, nf - 1u);
                for (unsigned j = j0; j <= j1; ++j) {
                    const unsigned b = off + (c * F + j) * bits;
                    const unsigned w = b >> 5, s = b & 31u;
                    uint32_t v = qs[w] >> s;
                    if (s + bits > 32u) v |= qs[w + 1] << (32u - s);
                    v &= mask;
                    const int d = (int)(j * bits) - (int)lo;
                    o |= d >= 0 ? v << d : v >> (-d);
                }
            }
            out[kk] = o;
        }
        dst[t] = make_uint4(out[0], out[1], out[2], out[3]);
    }
}

}  // namespace
}  // namespace eri

extern "C" eri_status_t eri_pack_paper512_stream(const void *d_stream, int64_t n_quartets,
                                                 int32_t n_eri, int32_t bits, void *d_chunks,
                                                 void *stream) {
    if (n_quartets < 0 || n_eri < 1 || n_eri > 50625 || bits < 2 || bits > 24) return ERI_E_INVALID;
    if (n_quartets == 0) return ERI_OK;
    if (!d_stream || !d_chunks) return ERI_E_INVALID;
    if (reinterpret_cast<uintptr_t>(d_stream) % 4 || reinterpret_cast<uintptr_t>(d_chunks) % 4)
        return ERI_E_INVALID;
    const long long F = 512 / bits;
    const long long n_cs = (n_eri + F - 1) / F;
    const long long per_piece = (1ll << 30) / (n_cs * eri::kChunkWords);  // >= 1: n_cs <= 50625
    const auto *src = static_cast<const uint32_t *>(d_stream);
    auto *dst = static_cast<uint32_t *>(d_chunks);
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return ERI_E_CUDA;
    const bool wide = reinterpret_cast<uintptr_t>(d_chunks) % 16 == 0;
    for (long long q0 = 0; q0 < n_quartets; q0 += per_piece) {
        const long long nq = n_quartets - q0 < per_piece ? n_quartets - q0 : per_piece;
        const long long words = nq * n_cs * eri::kChunkWords;
        long long blocks = ((wide ? words / 4 : words) + 255) / 256;
        if (blocks > 8ll * sms) blocks = 8ll * sms;  // grid-stride beyond 8 resident CTAs per SM
        if (wide)
            eri::paper512_kernel4<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
                src, (unsigned long long)q0, (unsigned)nq, (unsigned)n_eri, (unsigned)n_cs, (unsigned)bits,
                reinterpret_cast<uint4 *>(dst + q0 * n_cs * eri::kChunkWords));
        else
            eri::paper512_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
                src, (unsigned long long)q0, (unsigned)nq, (unsigned)n_eri, (unsigned)n_cs,
                (unsigned)bits, dst + q0 * n_cs * eri::kChunkWords);
        if (cudaGetLastError() != cudaSuccess) return ERI_E_CUDA;
    }
    return ERI_OK;
}
