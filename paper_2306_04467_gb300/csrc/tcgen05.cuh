// Fifth-generation tensor-core (tcgen05) building blocks for sm_103a, as
// inline PTX: tensor-memory allocation, the shared-memory matrix and
// instruction descriptors of a BF16 x BF16 -> FP32 MMA, the MMA itself, its
// completion on an mbarrier and the accumulator read-back.
//
// Operand layout (both A and B K-major, no swizzle): the matrix is cut into
// core matrices of 8 rows x 16 bytes (8 BF16), each stored as 8 contiguous
// 16-byte rows; core matrices adjacent along K lie kLbo bytes apart, core
// matrices adjacent along M (or N) kSbo bytes apart. With K = 32 (four core
// matrices along K, stored back to back) kLbo = 128 and kSbo = 512: element
// (r, k) of a tile sits at byte (r / 8) * 512 + (k / 8) * 128 + (r % 8) * 16
// + (k % 8) * 2.
#pragma once
#include <cstdint>

namespace gks2l {
namespace tc {

constexpr unsigned kLbo = 128, kSbo = 512;

// byte offset of element (r, k) of a [rows][32] BF16 operand tile
__host__ __device__ constexpr unsigned tile_offset(unsigned r, unsigned k) {
  return (r >> 3) * kSbo + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, all in 16-byte units; descriptor version 1; no swizzle.
__host__ __device__ constexpr uint64_t smem_desc(unsigned saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kLbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = m.
__host__ __device__ constexpr uint32_t idesc_bf16(unsigned m, unsigned n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

#ifdef __CUDACC__
__device__ __forceinline__ unsigned saddr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// allocate ncols tensor-memory columns (one full warp); the base address is
// written to *slot in shared memory
__device__ __forceinline__ void alloc(uint32_t *slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (tensor memory) = A B (+ D when accumulate), issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive on the mbarrier once every MMA this thread issued has completed
__device__ __forceinline__ void commit(void *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's shared-memory stores visible to the tensor cores
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of the warp's 32 lanes (lane i of the warp gets
// row 32 * (warp % 4) + i); taddr carries the warp's lane offset
__device__ __forceinline__ void ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}
#endif

}  // namespace tc
}  // namespace gks2l
