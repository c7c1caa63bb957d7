// The paper's output chunks (Sec. III-C, compress-store loops): every quartet's n-bit codes
// are written as 512-bit words of F = floor(512/n) fields; the fields that do not fit in one
// chunk open the next, the last chunk of a quartet is zero-padded, so a quartet takes
// n_CS = ceil(n_eri / F) chunks of 64 bytes and no chunk mixes quartets.  Field j of a chunk
// holds chunk bits [j*n, j*n + n), chunk bit s being bit s%32 of the chunk's 32-bit word s/32.
//
// The compressing kernels write the dense stream (every field right after the previous one);
// this file re-lays a class's dense stream into chunks.  It is integer-only, HBM-bound work.
// Because a quartet's fields are contiguous in the dense stream, chunk c of quartet i is the
// nf * n stream bits that start at bit (i * n_eri + c * F) * n, followed by zeros: every output
// word is a funnel shift of two neighbouring dense words, masked where the chunk's fields end,
// so no thread looks at individual fields.  Reads and writes are both coalesced along the chunk.
#include <cstdint>

#include <cuda_runtime.h>

#include "eri.h"

namespace eri {
namespace {

constexpr int kChunkWords = 16;  // 512 bits

// Output word `lo / 32` of a chunk whose first field starts at bit `s` of qs[w] (the word of
// the chunk bit lo) and whose fields fill `valid` bits.  A dense word is read only where it holds
// one of the chunk's bits, so nothing past the class's last code is read.
__device__ __forceinline__ uint32_t chunk_word(const uint32_t *__restrict__ qs, unsigned w, unsigned s,
                                               unsigned lo, unsigned valid) {
    if (lo >= valid) return 0u;
    const unsigned need = valid - lo;  // chunk bits left from lo on
    uint32_t v = qs[w] >> s;
    if (s + min(need, 32u) > 32u) v |= qs[w + 1] << (32u - s);  // s > 0 here
    if (need < 32u) v &= (1u << need) - 1u;
    return v;
}

// Quartets [q0, q0 + nq) of one class, one thread per output word.  `src` is the class's dense
// stream (word 0 holds stream bit 0), `dst` the chunk words of quartet q0.  nq * n_cs * 16 < 2^31
// (host-checked), and every in-quartet bit offset fits 32 bits (n_eri * bits <= 50625 * 24).
__global__ void __launch_bounds__(256) paper512_kernel(const uint32_t *__restrict__ src,
                                                       unsigned long long q0, unsigned nq,
                                                       unsigned n_eri, unsigned n_cs, unsigned bits,
                                                       uint32_t *__restrict__ dst) {
    const unsigned F = 512u / bits;
    const unsigned total = nq * n_cs * kChunkWords;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned ch = t / kChunkWords, k = t % kChunkWords;
        const unsigned i = ch / n_cs, c = ch - i * n_cs;
        const unsigned long long qbit = (q0 + i) * (unsigned long long)n_eri * bits;
        const uint32_t *qs = src + (qbit >> 5);
        const unsigned valid = min(F, n_eri - c * F) * bits;  // >= bits since c < n_cs
        const unsigned b = ((unsigned)qbit & 31u) + c * F * bits + 32u * k;
        dst[t] = chunk_word(qs, b >> 5, b & 31u, 32u * k, valid);
    }
}

// The same with one thread per quarter chunk: four consecutive output words share one shift
// and are written with one 16-byte store.  dst 16-byte aligned.
__global__ void __launch_bounds__(256) paper512_kernel4(const uint32_t *__restrict__ src,
                                                        unsigned long long q0, unsigned nq,
                                                        unsigned n_eri, unsigned n_cs, unsigned bits,
                                                        uint4 *__restrict__ dst) {
    const unsigned F = 512u / bits;
    const unsigned total = nq * n_cs * (kChunkWords / 4);
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned ch = t >> 2, lo = (t & 3u) * 128u;
        const unsigned i = ch / n_cs, c = ch - i * n_cs;
        const unsigned long long qbit = (q0 + i) * (unsigned long long)n_eri * bits;
        const uint32_t *qs = src + (qbit >> 5);
        const unsigned valid = min(F, n_eri - c * F) * bits;
        const unsigned b = ((unsigned)qbit & 31u) + c * F * bits + lo;
        const unsigned w = b >> 5, s = b & 31u;
        dst[t] = make_uint4(chunk_word(qs, w, s, lo, valid), chunk_word(qs, w + 1, s, lo + 32u, valid),
                            chunk_word(qs, w + 2, s, lo + 64u, valid), chunk_word(qs, w + 3, s, lo + 96u, valid));
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
