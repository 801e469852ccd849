// Double-float accumulation helpers shared by the cross-correlation and the
// per-bin-means kernels: error-free FP32 addition and a shared-memory
// histogram entry held as an unevaluated sum hi + lo of two floats.
#pragma once

#include "lya_internal.cuh"

namespace lya {

// s + e == a + b exactly (Knuth's TwoSum; no FMA contraction involved).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Retry limit of df_atomic_add: every failed swap means another thread's
// update went through, so the loop only ends here under a pathological
// interleaving; the entry is then left unchanged and FLAG_RETRY is raised.
constexpr int kDfRetry = 1 << 16;

// (hi, lo) pair at p (one 64-bit shared-memory word, hi in the low half)
// += h + l, renormalised so that |lo| stays below half an ulp of hi.
__device__ __forceinline__ void df_atomic_add(float2* p, float h, float l, unsigned* err) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(p);
  unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(a);
  for (int it = 0; it < kDfRetry; ++it) {
    float s, e;
    two_sum(__uint_as_float(static_cast<unsigned>(old)), h, s, e);
    const float t = __uint_as_float(static_cast<unsigned>(old >> 32)) + l + e;
    const float H = s + t;
    const float L = t - (H - s);
    const unsigned long long nw = static_cast<unsigned long long>(__float_as_uint(H)) |
                                  (static_cast<unsigned long long>(__float_as_uint(L)) << 32);
    const unsigned long long seen = atomicCAS(a, old, nw);
    if (seen == old) return;
    old = seen;
  }
  atomicOr(err, FLAG_RETRY);
}

// Barrier among the `threads` threads of one team of a block (named barrier
// `id` >= 1; id 0 is __syncthreads).
__device__ __forceinline__ void team_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

}  // namespace lya
