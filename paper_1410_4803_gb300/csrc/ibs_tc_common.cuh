// Building blocks of the tensor-core kernels (tcgen05): operand-tile layout,
// shared-memory and instruction descriptors, the MMA, commit and
// tensor-memory load wrappers, the unit scale factors of the block-scaled E2M1
// kind, and the bit-to-operand expansions.  Included by ibs_tc.cu (IBS pair
// counts) and ibs_ld.cu (LD correlation); each translation unit gets its own
// copy of these inline definitions.
//
// Operand tiles: 128 rows x 32 bytes (one MMA K step: 64 E2M1 or 32 E4M3
// values per row) in the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, the two core matrices of a row group 128 bytes apart
// (leading byte offset), row groups 256 bytes apart (stride byte offset).
// Rows 64..127 of a tile are its second contiguous 2 KiB, so a 64-row operand
// is half a tile.
#pragma once

#include <cstdint>

#include "ibs_device.cuh"
#include "ibs_internal.h"

namespace ibs {
namespace {

constexpr int kTB = 128;                          // samples per block (tile edge)
constexpr int kTileBytes = kTB * 32;              // one plane of one chunk: 128 rows x 32 bytes
constexpr uint32_t kTmemCols = 512;               // accumulators at 0/128/256, FP4 scale factors at 384..511
constexpr uint32_t kSfCol = 384;                  // scale factors of A at 384, of B at 448
constexpr uint8_t kFp8One = 0x38;                 // E4M3 1.0 (sign bit 0x80 makes -1.0)

// markers per chunk: one MMA K step
template <int F>
constexpr int kMarkers = F == kTcFp4 ? 64 : 32;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)(256 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version
  return d;                          // no swizzle
}

// Instruction descriptors, K-major A and B, M = 128.
// E4M3 x E4M3 -> F32 (kind::f8f6f4): D format F32 (bit 4), A and B formats
// E4M3 (0 at bits 7 and 10), N >> 3 at bit 17, M >> 4 at bit 24.
template <int N>
constexpr uint32_t kIdescFp8 = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
// Block-scaled E2M1 x E2M1 -> F32 (kind::mxf4): scale-factor ids 0 (bits 4
// and 29), A and B formats E2M1 (1 at bits 7 and 10), N >> 3 at bit 17, scale
// format UE8M0 (bit 23), M >> 4 at bit 24, K = 64.
template <int N>
constexpr uint32_t kIdescFp4 = (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) |
                               ((uint32_t)(128 >> 4) << 24);

// One MMA of the operand kind F, M = 128 and N columns; sf = the TMEM address
// of the scale factors (E2M1 only).
template <int F, int N = 128>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc, uint32_t sf) {
  if constexpr (F == kTcFp4) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n\t}" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(kIdescFp4<N>), "r"(acc), "r"(sf), "r"(sf + 64u)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdescFp8<N>), "r"(acc)
        : "memory");
  }
}

// FP4: every scale factor the MMAs can read is 1.0.  The calling warp fills
// its 32 TMEM lanes (quarter = warp % 4) at columns 384..511 with UE8M0 127
// bytes, so the factors read are 1.0 whichever byte and column of that range
// the hardware picks for a row.
__device__ __forceinline__ void tmem_fill_unit_scales(uint32_t tmem, int quarter) {
  const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + kSfCol;
  const uint32_t one = 0x7F7F7F7Fu;
#pragma unroll
  for (int c = 0; c < 128; c += 32)
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(base + c),
        "r"(one)
        : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

// Byte offset of (sample row r, byte column k) inside one 128 x 32-byte
// canonical tile (FP8: k is the marker; FP4: marker pair k holds markers 2k, 2k+1).
__device__ __forceinline__ int tile_off(int r, int k) {
  return (r >> 3) * 256 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15);
}

// ---------------------------------------------------------------------------
// Indicator bits -> operand bytes.  FP8: 4 bits become 4 bytes with a
// multiply, (x * 0x204081) & 0x01010101, and a second multiply makes each 1
// the E4M3 value.  FP4: 8 bits become 8 nibbles (bit t to bit 4t) by three
// shift-or-mask steps; E2M1 1.0 is 0b0010 and -1.0 is 0b1010.
__device__ __forceinline__ uint32_t spread4(uint32_t x) { return (x * 0x00204081u) & 0x01010101u; }

__device__ __forceinline__ uint32_t nib8(uint32_t x) {
  x &= 0xFFu;
  x = (x | (x << 12)) & 0x000F000Fu;
  x = (x | (x << 6)) & 0x03030303u;
  x = (x | (x << 3)) & 0x11111111u;
  return x;
}

}  // namespace
}  // namespace ibs
