// Complex float32 arithmetic and the 16-point DFT in registers, shared by the FFT kernels
// (Section 4, FFT pipelined with its inversion). A value is a float2 (re, im); transforms of sign
// S use the kernel W_M^(S n k) with W_M = e^(-2 pi i / M), so S = +1 is the forward DFT.
#pragma once

#include <cuda_runtime.h>

namespace mrw {
namespace fftk {

constexpr float kC8 = 0.92387953251128675613f;  // cos(pi / 8)
constexpr float kS8 = 0.38268343236508977173f;  // sin(pi / 8)
constexpr float kR2 = 0.70710678118654752440f;  // sqrt(1 / 2)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conj_if(float2 a, bool c) { return c ? make_float2(a.x, -a.y) : a; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -s i (the 4-point kernel W_4^s): s = +1 (forward) maps (x, y) to (y, -x)
template <int S>
__device__ __forceinline__ float2 rot(float2 a) {
  return S > 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// Sums and differences of both parts of a value at once (sm_100+ f32x2 instructions), rounded as
// the two float32 operations they replace.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long x, y, d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
  return r;
}

// 4-point DFT of (a, b, c, d) with kernel W_4^(S n k), results in place (index k). The sums and
// differences are paired instructions; -S i (b - d) is formed directly in its rotated order by two
// single subtractions, so no register swap is needed.
template <int S>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
  const float2 z0 = add2(a, c), z1 = sub2(a, c), z2 = add2(b, d);
  const float2 z3 = S > 0 ? make_float2(b.y - d.y, d.x - b.x) : make_float2(d.y - b.y, b.x - d.x);
  a = add2(z0, z2);
  c = sub2(z0, z2);
  b = add2(z1, z3);
  d = sub2(z1, z3);
}

// W_16^(S e) for the exponents the 4 x 4 split needs.
template <int S>
__device__ __forceinline__ float2 w16(int e) {
  const float s = (float)S;
  switch (e) {
    case 1: return make_float2(kC8, -s * kS8);
    case 2: return make_float2(kR2, -s * kR2);
    case 3: return make_float2(kS8, -s * kC8);
    case 4: return make_float2(0.f, -s);
    case 6: return make_float2(-kR2, -s * kR2);
    case 9: return make_float2(-kC8, s * kS8);
    default: return make_float2(1.f, 0.f);
  }
}

// 16-point DFT with kernel W_16^(S n k) of v[n]; the result X[k] is left in v[4 (k % 4) + k / 4].
template <int S>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<S>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);  // over n1
  // now v[4 k1 + n2] = y[k1][n2]; twiddle W_16^(n2 k1)
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)  // W_16^(4 S) = -S i is a rotation, not a multiplication
      v[4 * k1 + n2] = n2 * k1 == 4 ? rot<S>(v[4 * k1 + n2]) : cmul(v[4 * k1 + n2], w16<S>(n2 * k1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);  // over n2
}

__device__ __forceinline__ int dft16_slot(int k) { return 4 * (k & 3) + (k >> 2); }

}  // namespace fftk
}  // namespace mrw
