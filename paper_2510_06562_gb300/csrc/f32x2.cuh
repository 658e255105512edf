// Packed FP32 pair arithmetic of sm_100-family GPUs (PTX add/mul/fma with
// the .f32x2 type): one instruction applies the same IEEE single-precision
// operation, rounded to nearest even, to both halves of a 64-bit register
// pair. Each half's result equals the scalar operation's bit for bit, so
// code that pairs independent scalar operations this way keeps its results
// and halves the FP32 instructions it issues.
#pragma once

#include <stdint.h>

namespace dmts {
namespace f2 {

typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float lo(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}

__device__ __forceinline__ float hi(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}

__device__ __forceinline__ f32x2 splat(float x) { return pack(x, x); }

// a * b + c, a * b, a + b (each half)
__device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The two BF16 halves of a 32-bit word (low half first) as an exact FP32 pair.
__device__ __forceinline__ f32x2 from_bf16x2(uint32_t w) { return pack(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u)); }

}  // namespace f2
}  // namespace dmts
