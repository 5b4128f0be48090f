// tcgen05 helpers shared by the tensor-core kernels (inline PTX, sm_103a):
// fences, shared-memory matrix descriptors of the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; K-adjacent core
// matrices LBO bytes apart, 8-row groups SBO bytes apart), instruction
// descriptors, MMA issue, commit to an mbarrier, and TMEM loads.
#pragma once

#include "common.cuh"

namespace rp {
namespace {

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: no swizzle, LBO/SBO in bytes
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture
  return d;                 // base offset 0, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M as given
constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major
constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D (TMEM) [+]= A B^T with A (M x 8) and B (N x 8) TF32 in shared memory
__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 columns of FP32 from TMEM (one row per thread)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 head of an FP32 value: the 13 low mantissa bits cleared (exact in
// TF32); the tail x - head is the second term of the three-product split.
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Row `r` (K = NB values) of an operand array with `rows` rows in the
// no-swizzle K-major core-matrix layout (LBO = rows * 16 bytes, SBO = 128):
// element (r, k) at (k/4)*rows*16 + (r/8)*128 + (r%8)*16 + (k%4)*4.
template <int NB>
__device__ __forceinline__ void tc_put_row(unsigned char* arr, int rows, int r, const float (&v)[NB]) {
#pragma unroll
  for (int q = 0; q < NB / 4; ++q)
    *reinterpret_cast<float4*>(arr + q * rows * 16 + (r >> 3) * 128 + (r & 7) * 16) =
        make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// head and tail arrays of the real and imaginary parts of z[0..NB-1], at
// base, base + stride, base + 2 stride, base + 3 stride
template <int NB>
__device__ __forceinline__ void tc_put_split(unsigned char* base, uint32_t stride, int rows, int r,
                                             const c64 (&z)[NB]) {
  float h[NB], l[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    h[j] = tf32_head(z[j].re);
    l[j] = z[j].re - h[j];
  }
  tc_put_row<NB>(base, rows, r, h);
  tc_put_row<NB>(base + stride, rows, r, l);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    h[j] = tf32_head(z[j].im);
    l[j] = z[j].im - h[j];
  }
  tc_put_row<NB>(base + 2 * stride, rows, r, h);
  tc_put_row<NB>(base + 3 * stride, rows, r, l);
}

// columns 4 qq .. 4 qq + 3 of row r (z[0..3]) in the four split arrays of
// tc_put_split: one 16-byte core-matrix row in each
__device__ __forceinline__ void tc_put_split_quad(unsigned char* base, uint32_t stride, int rows, int r, int qq,
                                                  const c64 (&z)[4]) {
  unsigned char* p = base + qq * rows * 16 + (r >> 3) * 128 + (r & 7) * 16;
  float h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = tf32_head(z[j].re);
    l[j] = z[j].re - h[j];
  }
  *reinterpret_cast<float4*>(p) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(p + stride) = make_float4(l[0], l[1], l[2], l[3]);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = tf32_head(z[j].im);
    l[j] = z[j].im - h[j];
  }
  *reinterpret_cast<float4*>(p + 2 * stride) = make_float4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<float4*>(p + 3 * stride) = make_float4(l[0], l[1], l[2], l[3]);
}

// 32 lanes x 16 columns from each of two TMEM addresses, one wait
__device__ __forceinline__ void tc_ld16x2(uint32_t ta, uint32_t tb, float (&va)[16], float (&vb)[16]) {
  uint32_t a[16], c[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]),
        "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]), "=r"(c[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(a[i]);
    vb[i] = __uint_as_float(c[i]);
  }
}

}  // namespace
}  // namespace rp
