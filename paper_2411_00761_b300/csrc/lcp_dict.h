// lcp_dict.h -- launchers of the dictionary stage (k_dict.cu), internal.
//
// The last step of the paper's encoding stage is a dictionary coder (Sec.
// "Block coding", Zstd there).  This library's is an LZ77-style coder of a
// byte string -- normally a whole container -- into an "LCPZ" image:
//   0   "LCPZ", u8 version 1, u8 log2 chunk (16), u16 0
//   8   u64 raw bytes S, 16 u64 chunks C = ceil(S / 2^16), 24 u64 total T
//   32  the first min(S, 48) raw bytes, zero padded to 48 bytes (the
//       container header, readable without decoding)
//   80  u32 per chunk: its coded bytes, bit 31 set when stored raw
//   then zero padding to 16 bytes, the chunks back to back, padding to T.
// A chunk (2^16 bytes, the last one shorter) is coded alone as a list of
// sequences: a token byte (literal count << 4 | copy length - 4; a nibble of
// 15 is followed by an extension, bytes 255 ... 255 r added to it), the
// literal count's extension, the literals, and -- unless the chunk is
// complete after them -- a u16 little-endian copy offset and the copy
// length's extension.  Parse: every position i with four bytes left enters a
// 4096-entry table under the top 12 bits of (u32le(x[i..i+4)) * 2654435761
// mod 2^32), in order; the entry it replaces is its candidate; at the parse
// position a copy is taken when the candidate agrees on four bytes, as long
// as the bytes agree (to the chunk's end at most); otherwise one literal.  A
// chunk whose coding is not strictly shorter than its bytes is stored.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lcp {

constexpr uint32_t kDictLog2Chunk = 16;
constexpr uint64_t kDictHead = 80;

__host__ __device__ inline uint64_t dict_chunks(uint64_t raw) {
  return (raw + (1ull << kDictLog2Chunk) - 1) >> kDictLog2Chunk;
}
// first byte of the chunk bodies
__host__ __device__ inline uint64_t dict_body(uint64_t chunks) { return (kDictHead + 4 * chunks + 15) & ~15ull; }
// the image with every chunk stored
__host__ __device__ inline uint64_t dict_max_size(uint64_t raw) {
  return (dict_body(dict_chunks(raw)) + raw + 15) & ~15ull;
}

// codes every chunk of in[0, S) into scratch (chunk k at k * 2^16, S bytes)
// and writes its size-table entry sizes[k]
void launch_dict_encode(const uint8_t *in, uint64_t S, uint8_t *scratch, uint32_t *sizes, int sms,
                        cudaStream_t s);
// off[k] = dict_body(C) + the bytes of chunks 0..k-1 (entries masked of bit
// 31), k = 0..C; sizes is a device array of C entries (4-byte aligned)
void launch_dict_offsets(const uint32_t *sizes, uint64_t C, unsigned long long *off,
                         cudaStream_t s);
// the image (T bytes, T = off[C] rounded up to 16) of in[0, S) from the coded
// chunks in scratch; out 4-byte aligned, disjoint from in and scratch
void launch_dict_pack(const uint8_t *in, uint64_t S, const uint8_t *scratch, const uint32_t *sizes,
                      const unsigned long long *off, uint64_t T, uint8_t *out, int sms,
                      cudaStream_t s);
// decodes the chunks of an image (in_size bytes, header already checked:
// S, C, T <= in_size) into out[0, S); *err = 1 when a chunk or the size
// table is malformed (out is then unspecified)
void launch_dict_decode(const uint8_t *in, uint64_t in_size, uint64_t S, uint64_t T,
                        const unsigned long long *off, uint8_t *out, int *err, int sms,
                        cudaStream_t s);

}  // namespace lcp
