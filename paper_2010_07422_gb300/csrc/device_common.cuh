// Device helpers shared by the kernels of libircur.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ircur {

// splitmix64 output for state x (Steele, Lea, Flood, OOPSLA 2014): the
// finaliser applied to x + golden ratio, all arithmetic mod 2^64.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Index maps: entry i of a map holds index_tag(tag, a) when i is the a-th
// member of the index set of draw tag - 1 (positions below 2^9, draws below
// 2^23 - 1); entries of other draws carry other tags, 0 is no draw.
__host__ __device__ __forceinline__ unsigned index_tag(unsigned tag, int a) { return (tag << 9) | (unsigned)a; }
__host__ __device__ __forceinline__ bool index_tag_is(unsigned e, unsigned tag) { return (e >> 9) == tag; }
__host__ __device__ __forceinline__ int index_tag_pos(unsigned e) { return (int)(e & 511u); }

// The low-rank estimate at one entry, L_k(i,j) = A_k(i,:) B_k(:,j), as an FMA
// chain in the fixed order t = 0..R-1.  Every kernel that evaluates L_k at an
// entry of the (I,J) block uses this function, so the core, the row panel and
// the column panel see bit-identical values there.
template <int R>
__device__ __forceinline__ float lowrank_entry(const float* a, const float* b) {
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < R; ++t) acc = fmaf(a[t], b[t], acc);
  return acc;
}

// Two FMAs in one packed FP32 instruction (fma.rn.f32x2): d.x = fma(a.x, b.x,
// c.x), d.y = fma(a.y, b.y, c.y), each rounded to nearest like fmaf, so a
// chain of them gives, element by element, the values of the scalar chain.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ua, ub, uc, ud;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ua) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(ub) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(uc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(ud));
  return d;
}

// lowrank_entry for two columns at once: a broadcast to both, b0 and b1 the
// two columns; element for element the same FMA chain as lowrank_entry.
template <int R>
__device__ __forceinline__ float2 lowrank_entry2(const float* a, const float2* b) {
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < R; ++t) acc = ffma2(make_float2(a[t], a[t]), b[t], acc);
  return acc;
}

// BF16 storage of a panel entry (round to nearest even) and its value.
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf16_bits_to_f32(uint16_t h) { return __uint_as_float((unsigned)h << 16); }

// The precision variant's panel entry: the BF16 value, unless the threshold
// decision |d - l| > zeta could differ from the FP32 one.  Rounding to BF16
// moves d by at most 2^-9 |d| (8 significant bits, round to nearest), so the
// decisions agree whenever ||d_bf16 - l| - zeta| > 2^-8 |d_bf16| (a factor 2
// of margin); inside that band the FP32 entry is read (`exact`) and used.
template <typename F>
__device__ __forceinline__ float bf16_entry(uint16_t h, float l, float zeta, F exact) {
  const float d = bf16_bits_to_f32(h);
  if (fabsf(fabsf(d - l) - zeta) <= 0x1p-8f * fabsf(d) + 1e-30f) return exact();
  return d;
}

// One entry of D - S_{k+1} on a panel (Alg. 1, Phase I then Phase II):
// S = T_zeta(D - L_k) keeps the residual where |D - L_k| > zeta (Sec. 3.2,
// strict >), so D - S equals L_k there and D elsewhere.
__device__ __forceinline__ float panel_value(float d, float l, float zeta) {
  const float res = d - l;
  return fabsf(res) > zeta ? l : d;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- mbarrier / bulk-copy primitives (inline PTX, sm_90+ forms valid on sm_103a)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier: true when the phase
// completed, false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 1-D bulk copy global -> shared through the TMA engine, completing on an
// mbarrier.  dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only, no L1 allocation) and
// the wait for all of a thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// 4-byte asynchronous copy (any 4-byte aligned address).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: a primary grid lets the next kernel of the
// stream start once every CTA has executed launch_dependents (or exited); the
// dependent grid's griddepcontrol.wait blocks until the primary grid has
// completed and its memory operations are visible.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Nanosecond device clock (comparable across SMs).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Kernel-span trace: trace[slot] = earliest block start, trace[nslots + slot]
// = latest block end, in global_ns() units.  Null trace: no-op.
__device__ __forceinline__ void trace_start(unsigned long long* trace, int slot) {
  if (trace && threadIdx.x == 0) atomicMin(trace + slot, global_ns());
}
__device__ __forceinline__ void trace_stop(unsigned long long* trace, int nslots, int slot) {
  if (trace && threadIdx.x == 0) atomicMax(trace + nslots + slot, global_ns());
}

// Streaming 16-byte store (evict-first): outputs written once, never re-read here.
__device__ __forceinline__ void st_stream(float4* p, float4 v) { __stcs(p, v); }

}  // namespace ircur
