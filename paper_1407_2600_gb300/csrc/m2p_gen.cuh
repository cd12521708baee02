// Generated by gen_m2p.py -- do not edit by hand.
// Reduced-coefficient multipole-to-particle kernels, orders 0..4.
#pragma once

constexpr int kNB0 = 1;  // reduced coefficients at order 0
constexpr int kM2PFlops0 = 25;  // flops per M2P (FMA = 2, rsqrt = 1)
constexpr int kNB1 = 4;  // reduced coefficients at order 1
constexpr int kM2PFlops1 = 50;  // flops per M2P (FMA = 2, rsqrt = 1)
constexpr int kNB2 = 11;  // reduced coefficients at order 2
constexpr int kM2PFlops2 = 101;  // flops per M2P (FMA = 2, rsqrt = 1)
constexpr int kNB3 = 24;  // reduced coefficients at order 3
constexpr int kM2PFlops3 = 192;  // flops per M2P (FMA = 2, rsqrt = 1)
constexpr int kNB4 = 46;  // reduced coefficients at order 4
constexpr int kM2PFlops4 = 342;  // flops per M2P (FMA = 2, rsqrt = 1)

// REF: the reciprocal square root refined (near-uniform boxes), else the
// hardware approximation alone
template <typename T, bool REF = true>
__device__ __forceinline__ void m2p_p0(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                     T& ax, T& ay, T& az) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T m0 = T(1);
  T S0 = T(0), G0x = T(0), G0y = T(0), G0z = T(0);
  { const T b = B[0];
    S0 = fma(b, m0, S0);
  }
  T t = F1 * S0;
  ax = fma(Rx, t, ax);
  ay = fma(Ry, t, ay);
  az = fma(Rz, t, az);
}

template <typename T>
__device__ __forceinline__ T m2pot_p0(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  T S0 = T(0);
  S0 = S0 + B[0];
  return F0 * S0;
}

template <bool REF = true>
__device__ __forceinline__ void m2p2_p0(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz,
                                       float2 eps2, float2& ax, float2& ay, float2& az) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))
                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  float2 S0;
  { const float2 b = B[0];
    S0 = b;
  }
  float2 t = __fmul2_rn(F1, S0);
  ax = __ffma2_rn(Rx, t, ax);
  ay = __ffma2_rn(Ry, t, ay);
  az = __ffma2_rn(Rz, t, az);
}

__device__ __forceinline__ void reduce_moments_p0(const double* __restrict__ M, double* __restrict__ B) {
  B[0] = 1 * M[0];
}

// REF: the reciprocal square root refined (near-uniform boxes), else the
// hardware approximation alone
template <typename T, bool REF = true>
__device__ __forceinline__ void m2p_p1(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                     T& ax, T& ay, T& az) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T m0 = T(1);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  T S0 = T(0), G0x = T(0), G0y = T(0), G0z = T(0);
  T S1 = T(0), G1x = T(0), G1y = T(0), G1z = T(0);
  { const T b = B[0];
    S0 = fma(b, m0, S0);
  }
  { const T b = B[1];
    S1 = fma(b, m1, S1);
    G1x = fma(b, m0, G1x);
  }
  { const T b = B[2];
    S1 = fma(b, m2, S1);
    G1y = fma(b, m0, G1y);
  }
  { const T b = B[3];
    S1 = fma(b, m3, S1);
    G1z = fma(b, m0, G1z);
  }
  T t = F1 * S0;
  t = fma(F2, S1, t);
  ax = fma(Rx, t, fma(F1, G1x, ax));
  ay = fma(Ry, t, fma(F1, G1y, ay));
  az = fma(Rz, t, fma(F1, G1z, az));
}

template <typename T>
__device__ __forceinline__ T m2pot_p1(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  T S0 = T(0);
  T S1 = T(0);
  S0 = S0 + B[0];
  S1 = fma(B[1], m1, S1);
  S1 = fma(B[2], m2, S1);
  S1 = fma(B[3], m3, S1);
  return fma(F1, S1, F0 * S0);
}

template <bool REF = true>
__device__ __forceinline__ void m2p2_p1(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz,
                                       float2 eps2, float2& ax, float2& ay, float2& az) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))
                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 m1 = Rx;
  const float2 m2 = Ry;
  const float2 m3 = Rz;
  float2 S0, S1, G1x, G1y, G1z;
  { const float2 b = B[0];
    S0 = b;
  }
  { const float2 b = B[1];
    S1 = __fmul2_rn(b, m1);
    G1x = b;
  }
  { const float2 b = B[2];
    S1 = __ffma2_rn(b, m2, S1);
    G1y = b;
  }
  { const float2 b = B[3];
    S1 = __ffma2_rn(b, m3, S1);
    G1z = b;
  }
  float2 t = __fmul2_rn(F1, S0);
  t = __ffma2_rn(F2, S1, t);
  ax = __ffma2_rn(Rx, t, __ffma2_rn(F1, G1x, ax));
  ay = __ffma2_rn(Ry, t, __ffma2_rn(F1, G1y, ay));
  az = __ffma2_rn(Rz, t, __ffma2_rn(F1, G1z, az));
}

__device__ __forceinline__ void reduce_moments_p1(const double* __restrict__ M, double* __restrict__ B) {
  B[0] = 1 * M[0];
  B[1] = -1 * M[1];
  B[2] = -1 * M[2];
  B[3] = -1 * M[3];
}

// REF: the reciprocal square root refined (near-uniform boxes), else the
// hardware approximation alone
template <typename T, bool REF = true>
__device__ __forceinline__ void m2p_p2(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                     T& ax, T& ay, T& az) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Ry_2 = Ry * T(0.5);
  const T Rz_2 = Rz * T(0.5);
  const T m0 = T(1);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  T S0 = T(0), G0x = T(0), G0y = T(0), G0z = T(0);
  T S1 = T(0), G1x = T(0), G1y = T(0), G1z = T(0);
  T S2 = T(0), G2x = T(0), G2y = T(0), G2z = T(0);
  { const T b = B[0];
    S0 = fma(b, m0, S0);
  }
  { const T b = B[1];
    S1 = fma(b, m0, S1);
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = fma(b, m0, G1x);
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = fma(b, m0, G1y);
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = fma(b, m0, G1z);
  }
  { const T b = B[5];
    S2 = fma(b, m4, S2);
    G2x = fma(b, m1, G2x);
  }
  { const T b = B[6];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    G2y = fma(b, m1, G2y);
  }
  { const T b = B[7];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    G2z = fma(b, m1, G2z);
  }
  { const T b = B[8];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
  }
  { const T b = B[9];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    G2z = fma(b, m2, G2z);
  }
  { const T b = B[10];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
  }
  T t = F1 * S0;
  t = fma(F2, S1, t);
  t = fma(F3, S2, t);
  ax = fma(Rx, t, fma(F1, G1x, fma(F2, G2x, ax)));
  ay = fma(Ry, t, fma(F1, G1y, fma(F2, G2y, ay)));
  az = fma(Rz, t, fma(F1, G1z, fma(F2, G2z, az)));
}

template <typename T>
__device__ __forceinline__ T m2pot_p2(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Ry_2 = Ry * T(0.5);
  const T Rz_2 = Rz * T(0.5);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  T S0 = T(0);
  T S1 = T(0);
  T S2 = T(0);
  S0 = S0 + B[0];
  S1 = S1 + B[1];
  S1 = fma(B[2], m1, S1);
  S1 = fma(B[3], m2, S1);
  S1 = fma(B[4], m3, S1);
  S2 = fma(B[5], m4, S2);
  S2 = fma(B[6], m5, S2);
  S2 = fma(B[7], m6, S2);
  S2 = fma(B[8], m7, S2);
  S2 = fma(B[9], m8, S2);
  S2 = fma(B[10], m9, S2);
  return fma(F2, S2, fma(F1, S1, F0 * S0));
}

template <bool REF = true>
__device__ __forceinline__ void m2p2_p2(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz,
                                       float2 eps2, float2& ax, float2& ay, float2& az) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))
                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 m1 = Rx;
  const float2 m2 = Ry;
  const float2 m3 = Rz;
  const float2 m4 = __fmul2_rn(m1, Rx_2);
  const float2 m5 = __fmul2_rn(m2, Rx);
  const float2 m6 = __fmul2_rn(m3, Rx);
  const float2 m7 = __fmul2_rn(m2, Ry_2);
  const float2 m8 = __fmul2_rn(m3, Ry);
  const float2 m9 = __fmul2_rn(m3, Rz_2);
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z;
  { const float2 b = B[0];
    S0 = b;
  }
  { const float2 b = B[1];
    S1 = b;
  }
  { const float2 b = B[2];
    S1 = __ffma2_rn(b, m1, S1);
    G1x = b;
  }
  { const float2 b = B[3];
    S1 = __ffma2_rn(b, m2, S1);
    G1y = b;
  }
  { const float2 b = B[4];
    S1 = __ffma2_rn(b, m3, S1);
    G1z = b;
  }
  { const float2 b = B[5];
    S2 = __fmul2_rn(b, m4);
    G2x = __fmul2_rn(b, m1);
  }
  { const float2 b = B[6];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    G2y = __fmul2_rn(b, m1);
  }
  { const float2 b = B[7];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    G2z = __fmul2_rn(b, m1);
  }
  { const float2 b = B[8];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
  }
  { const float2 b = B[9];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    G2z = __ffma2_rn(b, m2, G2z);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
  }
  float2 t = __fmul2_rn(F1, S0);
  t = __ffma2_rn(F2, S1, t);
  t = __ffma2_rn(F3, S2, t);
  ax = __ffma2_rn(Rx, t, __ffma2_rn(F1, G1x, __ffma2_rn(F2, G2x, ax)));
  ay = __ffma2_rn(Ry, t, __ffma2_rn(F1, G1y, __ffma2_rn(F2, G2y, ay)));
  az = __ffma2_rn(Rz, t, __ffma2_rn(F1, G1z, __ffma2_rn(F2, G2z, az)));
}

__device__ __forceinline__ void reduce_moments_p2(const double* __restrict__ M, double* __restrict__ B) {
  B[0] = 1 * M[0];
  B[1] = 0.5 * M[4] + 0.5 * M[7] + 0.5 * M[9];
  B[2] = -1 * M[1];
  B[3] = -1 * M[2];
  B[4] = -1 * M[3];
  B[5] = 1 * M[4];
  B[6] = 1 * M[5];
  B[7] = 1 * M[6];
  B[8] = 1 * M[7];
  B[9] = 1 * M[8];
  B[10] = 1 * M[9];
}

// REF: the reciprocal square root refined (near-uniform boxes), else the
// hardware approximation alone
template <typename T, bool REF = true>
__device__ __forceinline__ void m2p_p3(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                     T& ax, T& ay, T& az) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Rx_3 = Rx * T(0.33333333333333331);
  const T Ry_2 = Ry * T(0.5);
  const T Ry_3 = Ry * T(0.33333333333333331);
  const T Rz_2 = Rz * T(0.5);
  const T Rz_3 = Rz * T(0.33333333333333331);
  const T m0 = T(1);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  const T m10 = m4 * Rx_3;
  const T m11 = m5 * Rx_2;
  const T m12 = m6 * Rx_2;
  const T m13 = m7 * Rx;
  const T m14 = m8 * Rx;
  const T m15 = m9 * Rx;
  const T m16 = m7 * Ry_3;
  const T m17 = m8 * Ry_2;
  const T m18 = m9 * Ry;
  const T m19 = m9 * Rz_3;
  T S0 = T(0), G0x = T(0), G0y = T(0), G0z = T(0);
  T S1 = T(0), G1x = T(0), G1y = T(0), G1z = T(0);
  T S2 = T(0), G2x = T(0), G2y = T(0), G2z = T(0);
  T S3 = T(0), G3x = T(0), G3y = T(0), G3z = T(0);
  { const T b = B[0];
    S0 = fma(b, m0, S0);
  }
  { const T b = B[1];
    S1 = fma(b, m0, S1);
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = fma(b, m0, G1x);
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = fma(b, m0, G1y);
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = fma(b, m0, G1z);
  }
  { const T b = B[5];
    S2 = fma(b, m1, S2);
    G2x = fma(b, m0, G2x);
  }
  { const T b = B[6];
    S2 = fma(b, m2, S2);
    G2y = fma(b, m0, G2y);
  }
  { const T b = B[7];
    S2 = fma(b, m3, S2);
    G2z = fma(b, m0, G2z);
  }
  { const T b = B[8];
    S2 = fma(b, m4, S2);
    G2x = fma(b, m1, G2x);
  }
  { const T b = B[9];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    G2y = fma(b, m1, G2y);
  }
  { const T b = B[10];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    G2z = fma(b, m1, G2z);
  }
  { const T b = B[11];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
  }
  { const T b = B[12];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    G2z = fma(b, m2, G2z);
  }
  { const T b = B[13];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
  }
  { const T b = B[14];
    S3 = fma(b, m10, S3);
    G3x = fma(b, m4, G3x);
  }
  { const T b = B[15];
    S3 = fma(b, m11, S3);
    G3x = fma(b, m5, G3x);
    G3y = fma(b, m4, G3y);
  }
  { const T b = B[16];
    S3 = fma(b, m12, S3);
    G3x = fma(b, m6, G3x);
    G3z = fma(b, m4, G3z);
  }
  { const T b = B[17];
    S3 = fma(b, m13, S3);
    G3x = fma(b, m7, G3x);
    G3y = fma(b, m5, G3y);
  }
  { const T b = B[18];
    S3 = fma(b, m14, S3);
    G3x = fma(b, m8, G3x);
    G3y = fma(b, m6, G3y);
    G3z = fma(b, m5, G3z);
  }
  { const T b = B[19];
    S3 = fma(b, m15, S3);
    G3x = fma(b, m9, G3x);
    G3z = fma(b, m6, G3z);
  }
  { const T b = B[20];
    S3 = fma(b, m16, S3);
    G3y = fma(b, m7, G3y);
  }
  { const T b = B[21];
    S3 = fma(b, m17, S3);
    G3y = fma(b, m8, G3y);
    G3z = fma(b, m7, G3z);
  }
  { const T b = B[22];
    S3 = fma(b, m18, S3);
    G3y = fma(b, m9, G3y);
    G3z = fma(b, m8, G3z);
  }
  { const T b = B[23];
    S3 = fma(b, m19, S3);
    G3z = fma(b, m9, G3z);
  }
  T t = F1 * S0;
  t = fma(F2, S1, t);
  t = fma(F3, S2, t);
  t = fma(F4, S3, t);
  ax = fma(Rx, t, fma(F1, G1x, fma(F2, G2x, fma(F3, G3x, ax))));
  ay = fma(Ry, t, fma(F1, G1y, fma(F2, G2y, fma(F3, G3y, ay))));
  az = fma(Rz, t, fma(F1, G1z, fma(F2, G2z, fma(F3, G3z, az))));
}

template <typename T>
__device__ __forceinline__ T m2pot_p3(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Rx_3 = Rx * T(0.33333333333333331);
  const T Ry_2 = Ry * T(0.5);
  const T Ry_3 = Ry * T(0.33333333333333331);
  const T Rz_2 = Rz * T(0.5);
  const T Rz_3 = Rz * T(0.33333333333333331);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  const T m10 = m4 * Rx_3;
  const T m11 = m5 * Rx_2;
  const T m12 = m6 * Rx_2;
  const T m13 = m7 * Rx;
  const T m14 = m8 * Rx;
  const T m15 = m9 * Rx;
  const T m16 = m7 * Ry_3;
  const T m17 = m8 * Ry_2;
  const T m18 = m9 * Ry;
  const T m19 = m9 * Rz_3;
  T S0 = T(0);
  T S1 = T(0);
  T S2 = T(0);
  T S3 = T(0);
  S0 = S0 + B[0];
  S1 = S1 + B[1];
  S1 = fma(B[2], m1, S1);
  S1 = fma(B[3], m2, S1);
  S1 = fma(B[4], m3, S1);
  S2 = fma(B[5], m1, S2);
  S2 = fma(B[6], m2, S2);
  S2 = fma(B[7], m3, S2);
  S2 = fma(B[8], m4, S2);
  S2 = fma(B[9], m5, S2);
  S2 = fma(B[10], m6, S2);
  S2 = fma(B[11], m7, S2);
  S2 = fma(B[12], m8, S2);
  S2 = fma(B[13], m9, S2);
  S3 = fma(B[14], m10, S3);
  S3 = fma(B[15], m11, S3);
  S3 = fma(B[16], m12, S3);
  S3 = fma(B[17], m13, S3);
  S3 = fma(B[18], m14, S3);
  S3 = fma(B[19], m15, S3);
  S3 = fma(B[20], m16, S3);
  S3 = fma(B[21], m17, S3);
  S3 = fma(B[22], m18, S3);
  S3 = fma(B[23], m19, S3);
  return fma(F3, S3, fma(F2, S2, fma(F1, S1, F0 * S0)));
}

template <bool REF = true>
__device__ __forceinline__ void m2p2_p3(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz,
                                       float2 eps2, float2& ax, float2& ay, float2& az) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))
                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 F4 = __fmul2_rn(F3, __fmul2_rn(make_float2(-7.0f, -7.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Rx_3 = __fmul2_rn(Rx, make_float2(0.333333333f, 0.333333333f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Ry_3 = __fmul2_rn(Ry, make_float2(0.333333333f, 0.333333333f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 Rz_3 = __fmul2_rn(Rz, make_float2(0.333333333f, 0.333333333f));
  const float2 m1 = Rx;
  const float2 m2 = Ry;
  const float2 m3 = Rz;
  const float2 m4 = __fmul2_rn(m1, Rx_2);
  const float2 m5 = __fmul2_rn(m2, Rx);
  const float2 m6 = __fmul2_rn(m3, Rx);
  const float2 m7 = __fmul2_rn(m2, Ry_2);
  const float2 m8 = __fmul2_rn(m3, Ry);
  const float2 m9 = __fmul2_rn(m3, Rz_2);
  const float2 m10 = __fmul2_rn(m4, Rx_3);
  const float2 m11 = __fmul2_rn(m5, Rx_2);
  const float2 m12 = __fmul2_rn(m6, Rx_2);
  const float2 m13 = __fmul2_rn(m7, Rx);
  const float2 m14 = __fmul2_rn(m8, Rx);
  const float2 m15 = __fmul2_rn(m9, Rx);
  const float2 m16 = __fmul2_rn(m7, Ry_3);
  const float2 m17 = __fmul2_rn(m8, Ry_2);
  const float2 m18 = __fmul2_rn(m9, Ry);
  const float2 m19 = __fmul2_rn(m9, Rz_3);
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, S3, G3x, G3y, G3z;
  { const float2 b = B[0];
    S0 = b;
  }
  { const float2 b = B[1];
    S1 = b;
  }
  { const float2 b = B[2];
    S1 = __ffma2_rn(b, m1, S1);
    G1x = b;
  }
  { const float2 b = B[3];
    S1 = __ffma2_rn(b, m2, S1);
    G1y = b;
  }
  { const float2 b = B[4];
    S1 = __ffma2_rn(b, m3, S1);
    G1z = b;
  }
  { const float2 b = B[5];
    S2 = __fmul2_rn(b, m1);
    G2x = b;
  }
  { const float2 b = B[6];
    S2 = __ffma2_rn(b, m2, S2);
    G2y = b;
  }
  { const float2 b = B[7];
    S2 = __ffma2_rn(b, m3, S2);
    G2z = b;
  }
  { const float2 b = B[8];
    S2 = __ffma2_rn(b, m4, S2);
    G2x = __ffma2_rn(b, m1, G2x);
  }
  { const float2 b = B[9];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    G2y = __ffma2_rn(b, m1, G2y);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    G2z = __ffma2_rn(b, m1, G2z);
  }
  { const float2 b = B[11];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
  }
  { const float2 b = B[12];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    G2z = __ffma2_rn(b, m2, G2z);
  }
  { const float2 b = B[13];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
  }
  { const float2 b = B[14];
    S3 = __fmul2_rn(b, m10);
    G3x = __fmul2_rn(b, m4);
  }
  { const float2 b = B[15];
    S3 = __ffma2_rn(b, m11, S3);
    G3x = __ffma2_rn(b, m5, G3x);
    G3y = __fmul2_rn(b, m4);
  }
  { const float2 b = B[16];
    S3 = __ffma2_rn(b, m12, S3);
    G3x = __ffma2_rn(b, m6, G3x);
    G3z = __fmul2_rn(b, m4);
  }
  { const float2 b = B[17];
    S3 = __ffma2_rn(b, m13, S3);
    G3x = __ffma2_rn(b, m7, G3x);
    G3y = __ffma2_rn(b, m5, G3y);
  }
  { const float2 b = B[18];
    S3 = __ffma2_rn(b, m14, S3);
    G3x = __ffma2_rn(b, m8, G3x);
    G3y = __ffma2_rn(b, m6, G3y);
    G3z = __ffma2_rn(b, m5, G3z);
  }
  { const float2 b = B[19];
    S3 = __ffma2_rn(b, m15, S3);
    G3x = __ffma2_rn(b, m9, G3x);
    G3z = __ffma2_rn(b, m6, G3z);
  }
  { const float2 b = B[20];
    S3 = __ffma2_rn(b, m16, S3);
    G3y = __ffma2_rn(b, m7, G3y);
  }
  { const float2 b = B[21];
    S3 = __ffma2_rn(b, m17, S3);
    G3y = __ffma2_rn(b, m8, G3y);
    G3z = __ffma2_rn(b, m7, G3z);
  }
  { const float2 b = B[22];
    S3 = __ffma2_rn(b, m18, S3);
    G3y = __ffma2_rn(b, m9, G3y);
    G3z = __ffma2_rn(b, m8, G3z);
  }
  { const float2 b = B[23];
    S3 = __ffma2_rn(b, m19, S3);
    G3z = __ffma2_rn(b, m9, G3z);
  }
  float2 t = __fmul2_rn(F1, S0);
  t = __ffma2_rn(F2, S1, t);
  t = __ffma2_rn(F3, S2, t);
  t = __ffma2_rn(F4, S3, t);
  ax = __ffma2_rn(Rx, t, __ffma2_rn(F1, G1x, __ffma2_rn(F2, G2x, __ffma2_rn(F3, G3x, ax))));
  ay = __ffma2_rn(Ry, t, __ffma2_rn(F1, G1y, __ffma2_rn(F2, G2y, __ffma2_rn(F3, G3y, ay))));
  az = __ffma2_rn(Rz, t, __ffma2_rn(F1, G1z, __ffma2_rn(F2, G2z, __ffma2_rn(F3, G3z, az))));
}

__device__ __forceinline__ void reduce_moments_p3(const double* __restrict__ M, double* __restrict__ B) {
  B[0] = 1 * M[0];
  B[1] = 0.5 * M[4] + 0.5 * M[7] + 0.5 * M[9];
  B[2] = -1 * M[1];
  B[3] = -1 * M[2];
  B[4] = -1 * M[3];
  B[5] = -0.5 * M[10] + -0.5 * M[13] + -0.5 * M[15];
  B[6] = -0.5 * M[11] + -0.5 * M[16] + -0.5 * M[18];
  B[7] = -0.5 * M[12] + -0.5 * M[17] + -0.5 * M[19];
  B[8] = 1 * M[4];
  B[9] = 1 * M[5];
  B[10] = 1 * M[6];
  B[11] = 1 * M[7];
  B[12] = 1 * M[8];
  B[13] = 1 * M[9];
  B[14] = -1 * M[10];
  B[15] = -1 * M[11];
  B[16] = -1 * M[12];
  B[17] = -1 * M[13];
  B[18] = -1 * M[14];
  B[19] = -1 * M[15];
  B[20] = -1 * M[16];
  B[21] = -1 * M[17];
  B[22] = -1 * M[18];
  B[23] = -1 * M[19];
}

// REF: the reciprocal square root refined (near-uniform boxes), else the
// hardware approximation alone
template <typename T, bool REF = true>
__device__ __forceinline__ void m2p_p4(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                     T& ax, T& ay, T& az) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = REF ? nbody_rsqrt(s) : nbody_rsqrt_pair(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T F5 = F4 * (T(-9) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Rx_3 = Rx * T(0.33333333333333331);
  const T Rx_4 = Rx * T(0.25);
  const T Ry_2 = Ry * T(0.5);
  const T Ry_3 = Ry * T(0.33333333333333331);
  const T Ry_4 = Ry * T(0.25);
  const T Rz_2 = Rz * T(0.5);
  const T Rz_3 = Rz * T(0.33333333333333331);
  const T Rz_4 = Rz * T(0.25);
  const T m0 = T(1);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  const T m10 = m4 * Rx_3;
  const T m11 = m5 * Rx_2;
  const T m12 = m6 * Rx_2;
  const T m13 = m7 * Rx;
  const T m14 = m8 * Rx;
  const T m15 = m9 * Rx;
  const T m16 = m7 * Ry_3;
  const T m17 = m8 * Ry_2;
  const T m18 = m9 * Ry;
  const T m19 = m9 * Rz_3;
  const T m20 = m10 * Rx_4;
  const T m21 = m11 * Rx_3;
  const T m22 = m12 * Rx_3;
  const T m23 = m13 * Rx_2;
  const T m24 = m14 * Rx_2;
  const T m25 = m15 * Rx_2;
  const T m26 = m16 * Rx;
  const T m27 = m17 * Rx;
  const T m28 = m18 * Rx;
  const T m29 = m19 * Rx;
  const T m30 = m16 * Ry_4;
  const T m31 = m17 * Ry_3;
  const T m32 = m18 * Ry_2;
  const T m33 = m19 * Ry;
  const T m34 = m19 * Rz_4;
  T S0 = T(0), G0x = T(0), G0y = T(0), G0z = T(0);
  T S1 = T(0), G1x = T(0), G1y = T(0), G1z = T(0);
  T S2 = T(0), G2x = T(0), G2y = T(0), G2z = T(0);
  T S3 = T(0), G3x = T(0), G3y = T(0), G3z = T(0);
  T S4 = T(0), G4x = T(0), G4y = T(0), G4z = T(0);
  { const T b = B[0];
    S0 = fma(b, m0, S0);
  }
  { const T b = B[1];
    S1 = fma(b, m0, S1);
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = fma(b, m0, G1x);
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = fma(b, m0, G1y);
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = fma(b, m0, G1z);
  }
  { const T b = B[5];
    S2 = fma(b, m0, S2);
  }
  { const T b = B[6];
    S2 = fma(b, m1, S2);
    G2x = fma(b, m0, G2x);
  }
  { const T b = B[7];
    S2 = fma(b, m2, S2);
    G2y = fma(b, m0, G2y);
  }
  { const T b = B[8];
    S2 = fma(b, m3, S2);
    G2z = fma(b, m0, G2z);
  }
  { const T b = B[9];
    S2 = fma(b, m4, S2);
    G2x = fma(b, m1, G2x);
  }
  { const T b = B[10];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    G2y = fma(b, m1, G2y);
  }
  { const T b = B[11];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    G2z = fma(b, m1, G2z);
  }
  { const T b = B[12];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
  }
  { const T b = B[13];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    G2z = fma(b, m2, G2z);
  }
  { const T b = B[14];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
  }
  { const T b = B[15];
    S3 = fma(b, m4, S3);
    G3x = fma(b, m1, G3x);
  }
  { const T b = B[16];
    S3 = fma(b, m5, S3);
    G3x = fma(b, m2, G3x);
    G3y = fma(b, m1, G3y);
  }
  { const T b = B[17];
    S3 = fma(b, m6, S3);
    G3x = fma(b, m3, G3x);
    G3z = fma(b, m1, G3z);
  }
  { const T b = B[18];
    S3 = fma(b, m7, S3);
    G3y = fma(b, m2, G3y);
  }
  { const T b = B[19];
    S3 = fma(b, m8, S3);
    G3y = fma(b, m3, G3y);
    G3z = fma(b, m2, G3z);
  }
  { const T b = B[20];
    S3 = fma(b, m9, S3);
    G3z = fma(b, m3, G3z);
  }
  { const T b = B[21];
    S3 = fma(b, m10, S3);
    G3x = fma(b, m4, G3x);
  }
  { const T b = B[22];
    S3 = fma(b, m11, S3);
    G3x = fma(b, m5, G3x);
    G3y = fma(b, m4, G3y);
  }
  { const T b = B[23];
    S3 = fma(b, m12, S3);
    G3x = fma(b, m6, G3x);
    G3z = fma(b, m4, G3z);
  }
  { const T b = B[24];
    S3 = fma(b, m13, S3);
    G3x = fma(b, m7, G3x);
    G3y = fma(b, m5, G3y);
  }
  { const T b = B[25];
    S3 = fma(b, m14, S3);
    G3x = fma(b, m8, G3x);
    G3y = fma(b, m6, G3y);
    G3z = fma(b, m5, G3z);
  }
  { const T b = B[26];
    S3 = fma(b, m15, S3);
    G3x = fma(b, m9, G3x);
    G3z = fma(b, m6, G3z);
  }
  { const T b = B[27];
    S3 = fma(b, m16, S3);
    G3y = fma(b, m7, G3y);
  }
  { const T b = B[28];
    S3 = fma(b, m17, S3);
    G3y = fma(b, m8, G3y);
    G3z = fma(b, m7, G3z);
  }
  { const T b = B[29];
    S3 = fma(b, m18, S3);
    G3y = fma(b, m9, G3y);
    G3z = fma(b, m8, G3z);
  }
  { const T b = B[30];
    S3 = fma(b, m19, S3);
    G3z = fma(b, m9, G3z);
  }
  { const T b = B[31];
    S4 = fma(b, m20, S4);
    G4x = fma(b, m10, G4x);
  }
  { const T b = B[32];
    S4 = fma(b, m21, S4);
    G4x = fma(b, m11, G4x);
    G4y = fma(b, m10, G4y);
  }
  { const T b = B[33];
    S4 = fma(b, m22, S4);
    G4x = fma(b, m12, G4x);
    G4z = fma(b, m10, G4z);
  }
  { const T b = B[34];
    S4 = fma(b, m23, S4);
    G4x = fma(b, m13, G4x);
    G4y = fma(b, m11, G4y);
  }
  { const T b = B[35];
    S4 = fma(b, m24, S4);
    G4x = fma(b, m14, G4x);
    G4y = fma(b, m12, G4y);
    G4z = fma(b, m11, G4z);
  }
  { const T b = B[36];
    S4 = fma(b, m25, S4);
    G4x = fma(b, m15, G4x);
    G4z = fma(b, m12, G4z);
  }
  { const T b = B[37];
    S4 = fma(b, m26, S4);
    G4x = fma(b, m16, G4x);
    G4y = fma(b, m13, G4y);
  }
  { const T b = B[38];
    S4 = fma(b, m27, S4);
    G4x = fma(b, m17, G4x);
    G4y = fma(b, m14, G4y);
    G4z = fma(b, m13, G4z);
  }
  { const T b = B[39];
    S4 = fma(b, m28, S4);
    G4x = fma(b, m18, G4x);
    G4y = fma(b, m15, G4y);
    G4z = fma(b, m14, G4z);
  }
  { const T b = B[40];
    S4 = fma(b, m29, S4);
    G4x = fma(b, m19, G4x);
    G4z = fma(b, m15, G4z);
  }
  { const T b = B[41];
    S4 = fma(b, m30, S4);
    G4y = fma(b, m16, G4y);
  }
  { const T b = B[42];
    S4 = fma(b, m31, S4);
    G4y = fma(b, m17, G4y);
    G4z = fma(b, m16, G4z);
  }
  { const T b = B[43];
    S4 = fma(b, m32, S4);
    G4y = fma(b, m18, G4y);
    G4z = fma(b, m17, G4z);
  }
  { const T b = B[44];
    S4 = fma(b, m33, S4);
    G4y = fma(b, m19, G4y);
    G4z = fma(b, m18, G4z);
  }
  { const T b = B[45];
    S4 = fma(b, m34, S4);
    G4z = fma(b, m19, G4z);
  }
  T t = F1 * S0;
  t = fma(F2, S1, t);
  t = fma(F3, S2, t);
  t = fma(F4, S3, t);
  t = fma(F5, S4, t);
  ax = fma(Rx, t, fma(F1, G1x, fma(F2, G2x, fma(F3, G3x, fma(F4, G4x, ax)))));
  ay = fma(Ry, t, fma(F1, G1y, fma(F2, G2y, fma(F3, G3y, fma(F4, G4y, ay)))));
  az = fma(Rz, t, fma(F1, G1z, fma(F2, G2z, fma(F3, G3z, fma(F4, G4z, az)))));
}

template <typename T>
__device__ __forceinline__ T m2pot_p4(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T Rx_2 = Rx * T(0.5);
  const T Rx_3 = Rx * T(0.33333333333333331);
  const T Rx_4 = Rx * T(0.25);
  const T Ry_2 = Ry * T(0.5);
  const T Ry_3 = Ry * T(0.33333333333333331);
  const T Ry_4 = Ry * T(0.25);
  const T Rz_2 = Rz * T(0.5);
  const T Rz_3 = Rz * T(0.33333333333333331);
  const T Rz_4 = Rz * T(0.25);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  const T m4 = m1 * Rx_2;
  const T m5 = m2 * Rx;
  const T m6 = m3 * Rx;
  const T m7 = m2 * Ry_2;
  const T m8 = m3 * Ry;
  const T m9 = m3 * Rz_2;
  const T m10 = m4 * Rx_3;
  const T m11 = m5 * Rx_2;
  const T m12 = m6 * Rx_2;
  const T m13 = m7 * Rx;
  const T m14 = m8 * Rx;
  const T m15 = m9 * Rx;
  const T m16 = m7 * Ry_3;
  const T m17 = m8 * Ry_2;
  const T m18 = m9 * Ry;
  const T m19 = m9 * Rz_3;
  const T m20 = m10 * Rx_4;
  const T m21 = m11 * Rx_3;
  const T m22 = m12 * Rx_3;
  const T m23 = m13 * Rx_2;
  const T m24 = m14 * Rx_2;
  const T m25 = m15 * Rx_2;
  const T m26 = m16 * Rx;
  const T m27 = m17 * Rx;
  const T m28 = m18 * Rx;
  const T m29 = m19 * Rx;
  const T m30 = m16 * Ry_4;
  const T m31 = m17 * Ry_3;
  const T m32 = m18 * Ry_2;
  const T m33 = m19 * Ry;
  const T m34 = m19 * Rz_4;
  T S0 = T(0);
  T S1 = T(0);
  T S2 = T(0);
  T S3 = T(0);
  T S4 = T(0);
  S0 = S0 + B[0];
  S1 = S1 + B[1];
  S1 = fma(B[2], m1, S1);
  S1 = fma(B[3], m2, S1);
  S1 = fma(B[4], m3, S1);
  S2 = S2 + B[5];
  S2 = fma(B[6], m1, S2);
  S2 = fma(B[7], m2, S2);
  S2 = fma(B[8], m3, S2);
  S2 = fma(B[9], m4, S2);
  S2 = fma(B[10], m5, S2);
  S2 = fma(B[11], m6, S2);
  S2 = fma(B[12], m7, S2);
  S2 = fma(B[13], m8, S2);
  S2 = fma(B[14], m9, S2);
  S3 = fma(B[15], m4, S3);
  S3 = fma(B[16], m5, S3);
  S3 = fma(B[17], m6, S3);
  S3 = fma(B[18], m7, S3);
  S3 = fma(B[19], m8, S3);
  S3 = fma(B[20], m9, S3);
  S3 = fma(B[21], m10, S3);
  S3 = fma(B[22], m11, S3);
  S3 = fma(B[23], m12, S3);
  S3 = fma(B[24], m13, S3);
  S3 = fma(B[25], m14, S3);
  S3 = fma(B[26], m15, S3);
  S3 = fma(B[27], m16, S3);
  S3 = fma(B[28], m17, S3);
  S3 = fma(B[29], m18, S3);
  S3 = fma(B[30], m19, S3);
  S4 = fma(B[31], m20, S4);
  S4 = fma(B[32], m21, S4);
  S4 = fma(B[33], m22, S4);
  S4 = fma(B[34], m23, S4);
  S4 = fma(B[35], m24, S4);
  S4 = fma(B[36], m25, S4);
  S4 = fma(B[37], m26, S4);
  S4 = fma(B[38], m27, S4);
  S4 = fma(B[39], m28, S4);
  S4 = fma(B[40], m29, S4);
  S4 = fma(B[41], m30, S4);
  S4 = fma(B[42], m31, S4);
  S4 = fma(B[43], m32, S4);
  S4 = fma(B[44], m33, S4);
  S4 = fma(B[45], m34, S4);
  return fma(F4, S4, fma(F3, S3, fma(F2, S2, fma(F1, S1, F0 * S0))));
}

template <bool REF = true>
__device__ __forceinline__ void m2p2_p4(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz,
                                       float2 eps2, float2& ax, float2& ay, float2& az) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = REF ? make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y))
                        : make_float2(nbody_rsqrt_pair(s.x), nbody_rsqrt_pair(s.y));
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 F4 = __fmul2_rn(F3, __fmul2_rn(make_float2(-7.0f, -7.0f), is));
  const float2 F5 = __fmul2_rn(F4, __fmul2_rn(make_float2(-9.0f, -9.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Rx_3 = __fmul2_rn(Rx, make_float2(0.333333333f, 0.333333333f));
  const float2 Rx_4 = __fmul2_rn(Rx, make_float2(0.25f, 0.25f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Ry_3 = __fmul2_rn(Ry, make_float2(0.333333333f, 0.333333333f));
  const float2 Ry_4 = __fmul2_rn(Ry, make_float2(0.25f, 0.25f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 Rz_3 = __fmul2_rn(Rz, make_float2(0.333333333f, 0.333333333f));
  const float2 Rz_4 = __fmul2_rn(Rz, make_float2(0.25f, 0.25f));
  const float2 m1 = Rx;
  const float2 m2 = Ry;
  const float2 m3 = Rz;
  const float2 m4 = __fmul2_rn(m1, Rx_2);
  const float2 m5 = __fmul2_rn(m2, Rx);
  const float2 m6 = __fmul2_rn(m3, Rx);
  const float2 m7 = __fmul2_rn(m2, Ry_2);
  const float2 m8 = __fmul2_rn(m3, Ry);
  const float2 m9 = __fmul2_rn(m3, Rz_2);
  const float2 m10 = __fmul2_rn(m4, Rx_3);
  const float2 m11 = __fmul2_rn(m5, Rx_2);
  const float2 m12 = __fmul2_rn(m6, Rx_2);
  const float2 m13 = __fmul2_rn(m7, Rx);
  const float2 m14 = __fmul2_rn(m8, Rx);
  const float2 m15 = __fmul2_rn(m9, Rx);
  const float2 m16 = __fmul2_rn(m7, Ry_3);
  const float2 m17 = __fmul2_rn(m8, Ry_2);
  const float2 m18 = __fmul2_rn(m9, Ry);
  const float2 m19 = __fmul2_rn(m9, Rz_3);
  const float2 m20 = __fmul2_rn(m10, Rx_4);
  const float2 m21 = __fmul2_rn(m11, Rx_3);
  const float2 m22 = __fmul2_rn(m12, Rx_3);
  const float2 m23 = __fmul2_rn(m13, Rx_2);
  const float2 m24 = __fmul2_rn(m14, Rx_2);
  const float2 m25 = __fmul2_rn(m15, Rx_2);
  const float2 m26 = __fmul2_rn(m16, Rx);
  const float2 m27 = __fmul2_rn(m17, Rx);
  const float2 m28 = __fmul2_rn(m18, Rx);
  const float2 m29 = __fmul2_rn(m19, Rx);
  const float2 m30 = __fmul2_rn(m16, Ry_4);
  const float2 m31 = __fmul2_rn(m17, Ry_3);
  const float2 m32 = __fmul2_rn(m18, Ry_2);
  const float2 m33 = __fmul2_rn(m19, Ry);
  const float2 m34 = __fmul2_rn(m19, Rz_4);
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, S3, G3x, G3y, G3z, S4, G4x, G4y, G4z;
  { const float2 b = B[0];
    S0 = b;
  }
  { const float2 b = B[1];
    S1 = b;
  }
  { const float2 b = B[2];
    S1 = __ffma2_rn(b, m1, S1);
    G1x = b;
  }
  { const float2 b = B[3];
    S1 = __ffma2_rn(b, m2, S1);
    G1y = b;
  }
  { const float2 b = B[4];
    S1 = __ffma2_rn(b, m3, S1);
    G1z = b;
  }
  { const float2 b = B[5];
    S2 = b;
  }
  { const float2 b = B[6];
    S2 = __ffma2_rn(b, m1, S2);
    G2x = b;
  }
  { const float2 b = B[7];
    S2 = __ffma2_rn(b, m2, S2);
    G2y = b;
  }
  { const float2 b = B[8];
    S2 = __ffma2_rn(b, m3, S2);
    G2z = b;
  }
  { const float2 b = B[9];
    S2 = __ffma2_rn(b, m4, S2);
    G2x = __ffma2_rn(b, m1, G2x);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    G2y = __ffma2_rn(b, m1, G2y);
  }
  { const float2 b = B[11];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    G2z = __ffma2_rn(b, m1, G2z);
  }
  { const float2 b = B[12];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
  }
  { const float2 b = B[13];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    G2z = __ffma2_rn(b, m2, G2z);
  }
  { const float2 b = B[14];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
  }
  { const float2 b = B[15];
    S3 = __fmul2_rn(b, m4);
    G3x = __fmul2_rn(b, m1);
  }
  { const float2 b = B[16];
    S3 = __ffma2_rn(b, m5, S3);
    G3x = __ffma2_rn(b, m2, G3x);
    G3y = __fmul2_rn(b, m1);
  }
  { const float2 b = B[17];
    S3 = __ffma2_rn(b, m6, S3);
    G3x = __ffma2_rn(b, m3, G3x);
    G3z = __fmul2_rn(b, m1);
  }
  { const float2 b = B[18];
    S3 = __ffma2_rn(b, m7, S3);
    G3y = __ffma2_rn(b, m2, G3y);
  }
  { const float2 b = B[19];
    S3 = __ffma2_rn(b, m8, S3);
    G3y = __ffma2_rn(b, m3, G3y);
    G3z = __ffma2_rn(b, m2, G3z);
  }
  { const float2 b = B[20];
    S3 = __ffma2_rn(b, m9, S3);
    G3z = __ffma2_rn(b, m3, G3z);
  }
  { const float2 b = B[21];
    S3 = __ffma2_rn(b, m10, S3);
    G3x = __ffma2_rn(b, m4, G3x);
  }
  { const float2 b = B[22];
    S3 = __ffma2_rn(b, m11, S3);
    G3x = __ffma2_rn(b, m5, G3x);
    G3y = __ffma2_rn(b, m4, G3y);
  }
  { const float2 b = B[23];
    S3 = __ffma2_rn(b, m12, S3);
    G3x = __ffma2_rn(b, m6, G3x);
    G3z = __ffma2_rn(b, m4, G3z);
  }
  { const float2 b = B[24];
    S3 = __ffma2_rn(b, m13, S3);
    G3x = __ffma2_rn(b, m7, G3x);
    G3y = __ffma2_rn(b, m5, G3y);
  }
  { const float2 b = B[25];
    S3 = __ffma2_rn(b, m14, S3);
    G3x = __ffma2_rn(b, m8, G3x);
    G3y = __ffma2_rn(b, m6, G3y);
    G3z = __ffma2_rn(b, m5, G3z);
  }
  { const float2 b = B[26];
    S3 = __ffma2_rn(b, m15, S3);
    G3x = __ffma2_rn(b, m9, G3x);
    G3z = __ffma2_rn(b, m6, G3z);
  }
  { const float2 b = B[27];
    S3 = __ffma2_rn(b, m16, S3);
    G3y = __ffma2_rn(b, m7, G3y);
  }
  { const float2 b = B[28];
    S3 = __ffma2_rn(b, m17, S3);
    G3y = __ffma2_rn(b, m8, G3y);
    G3z = __ffma2_rn(b, m7, G3z);
  }
  { const float2 b = B[29];
    S3 = __ffma2_rn(b, m18, S3);
    G3y = __ffma2_rn(b, m9, G3y);
    G3z = __ffma2_rn(b, m8, G3z);
  }
  { const float2 b = B[30];
    S3 = __ffma2_rn(b, m19, S3);
    G3z = __ffma2_rn(b, m9, G3z);
  }
  { const float2 b = B[31];
    S4 = __fmul2_rn(b, m20);
    G4x = __fmul2_rn(b, m10);
  }
  { const float2 b = B[32];
    S4 = __ffma2_rn(b, m21, S4);
    G4x = __ffma2_rn(b, m11, G4x);
    G4y = __fmul2_rn(b, m10);
  }
  { const float2 b = B[33];
    S4 = __ffma2_rn(b, m22, S4);
    G4x = __ffma2_rn(b, m12, G4x);
    G4z = __fmul2_rn(b, m10);
  }
  { const float2 b = B[34];
    S4 = __ffma2_rn(b, m23, S4);
    G4x = __ffma2_rn(b, m13, G4x);
    G4y = __ffma2_rn(b, m11, G4y);
  }
  { const float2 b = B[35];
    S4 = __ffma2_rn(b, m24, S4);
    G4x = __ffma2_rn(b, m14, G4x);
    G4y = __ffma2_rn(b, m12, G4y);
    G4z = __ffma2_rn(b, m11, G4z);
  }
  { const float2 b = B[36];
    S4 = __ffma2_rn(b, m25, S4);
    G4x = __ffma2_rn(b, m15, G4x);
    G4z = __ffma2_rn(b, m12, G4z);
  }
  { const float2 b = B[37];
    S4 = __ffma2_rn(b, m26, S4);
    G4x = __ffma2_rn(b, m16, G4x);
    G4y = __ffma2_rn(b, m13, G4y);
  }
  { const float2 b = B[38];
    S4 = __ffma2_rn(b, m27, S4);
    G4x = __ffma2_rn(b, m17, G4x);
    G4y = __ffma2_rn(b, m14, G4y);
    G4z = __ffma2_rn(b, m13, G4z);
  }
  { const float2 b = B[39];
    S4 = __ffma2_rn(b, m28, S4);
    G4x = __ffma2_rn(b, m18, G4x);
    G4y = __ffma2_rn(b, m15, G4y);
    G4z = __ffma2_rn(b, m14, G4z);
  }
  { const float2 b = B[40];
    S4 = __ffma2_rn(b, m29, S4);
    G4x = __ffma2_rn(b, m19, G4x);
    G4z = __ffma2_rn(b, m15, G4z);
  }
  { const float2 b = B[41];
    S4 = __ffma2_rn(b, m30, S4);
    G4y = __ffma2_rn(b, m16, G4y);
  }
  { const float2 b = B[42];
    S4 = __ffma2_rn(b, m31, S4);
    G4y = __ffma2_rn(b, m17, G4y);
    G4z = __ffma2_rn(b, m16, G4z);
  }
  { const float2 b = B[43];
    S4 = __ffma2_rn(b, m32, S4);
    G4y = __ffma2_rn(b, m18, G4y);
    G4z = __ffma2_rn(b, m17, G4z);
  }
  { const float2 b = B[44];
    S4 = __ffma2_rn(b, m33, S4);
    G4y = __ffma2_rn(b, m19, G4y);
    G4z = __ffma2_rn(b, m18, G4z);
  }
  { const float2 b = B[45];
    S4 = __ffma2_rn(b, m34, S4);
    G4z = __ffma2_rn(b, m19, G4z);
  }
  float2 t = __fmul2_rn(F1, S0);
  t = __ffma2_rn(F2, S1, t);
  t = __ffma2_rn(F3, S2, t);
  t = __ffma2_rn(F4, S3, t);
  t = __ffma2_rn(F5, S4, t);
  ax = __ffma2_rn(Rx, t, __ffma2_rn(F1, G1x, __ffma2_rn(F2, G2x, __ffma2_rn(F3, G3x, __ffma2_rn(F4, G4x, ax)))));
  ay = __ffma2_rn(Ry, t, __ffma2_rn(F1, G1y, __ffma2_rn(F2, G2y, __ffma2_rn(F3, G3y, __ffma2_rn(F4, G4y, ay)))));
  az = __ffma2_rn(Rz, t, __ffma2_rn(F1, G1z, __ffma2_rn(F2, G2z, __ffma2_rn(F3, G3z, __ffma2_rn(F4, G4z, az)))));
}

__device__ __forceinline__ void reduce_moments_p4(const double* __restrict__ M, double* __restrict__ B) {
  B[0] = 1 * M[0];
  B[1] = 0.5 * M[4] + 0.5 * M[7] + 0.5 * M[9];
  B[2] = -1 * M[1];
  B[3] = -1 * M[2];
  B[4] = -1 * M[3];
  B[5] = 0.125 * M[20] + 0.25 * M[23] + 0.25 * M[25] + 0.125 * M[30] + 0.25 * M[32] + 0.125 * M[34];
  B[6] = -0.5 * M[10] + -0.5 * M[13] + -0.5 * M[15];
  B[7] = -0.5 * M[11] + -0.5 * M[16] + -0.5 * M[18];
  B[8] = -0.5 * M[12] + -0.5 * M[17] + -0.5 * M[19];
  B[9] = 1 * M[4];
  B[10] = 1 * M[5];
  B[11] = 1 * M[6];
  B[12] = 1 * M[7];
  B[13] = 1 * M[8];
  B[14] = 1 * M[9];
  B[15] = 0.5 * M[20] + 0.5 * M[23] + 0.5 * M[25];
  B[16] = 0.5 * M[21] + 0.5 * M[26] + 0.5 * M[28];
  B[17] = 0.5 * M[22] + 0.5 * M[27] + 0.5 * M[29];
  B[18] = 0.5 * M[23] + 0.5 * M[30] + 0.5 * M[32];
  B[19] = 0.5 * M[24] + 0.5 * M[31] + 0.5 * M[33];
  B[20] = 0.5 * M[25] + 0.5 * M[32] + 0.5 * M[34];
  B[21] = -1 * M[10];
  B[22] = -1 * M[11];
  B[23] = -1 * M[12];
  B[24] = -1 * M[13];
  B[25] = -1 * M[14];
  B[26] = -1 * M[15];
  B[27] = -1 * M[16];
  B[28] = -1 * M[17];
  B[29] = -1 * M[18];
  B[30] = -1 * M[19];
  B[31] = 1 * M[20];
  B[32] = 1 * M[21];
  B[33] = 1 * M[22];
  B[34] = 1 * M[23];
  B[35] = 1 * M[24];
  B[36] = 1 * M[25];
  B[37] = 1 * M[26];
  B[38] = 1 * M[27];
  B[39] = 1 * M[28];
  B[40] = 1 * M[29];
  B[41] = 1 * M[30];
  B[42] = 1 * M[31];
  B[43] = 1 * M[32];
  B[44] = 1 * M[33];
  B[45] = 1 * M[34];
}

__device__ __forceinline__ void p2m_acc_p0(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
}

__device__ __forceinline__ void m2m_acc_p0(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
}

__device__ __forceinline__ void p2m_acc_p1(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
  const double q1 = q0 * dx;
  M[1] += q1;
  const double q2 = q0 * dy;
  M[2] += q2;
  const double q3 = q0 * dz;
  M[3] += q3;
}

__device__ __forceinline__ void m2m_acc_p1(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
  Mp[1] = fma(w0, Mc[1], fma(w1, Mc[0], Mp[1]));
  Mp[2] = fma(w0, Mc[2], fma(w2, Mc[0], Mp[2]));
  Mp[3] = fma(w0, Mc[3], fma(w3, Mc[0], Mp[3]));
}

__device__ __forceinline__ void p2m_acc_p2(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
  const double q1 = q0 * dx;
  M[1] += q1;
  const double q2 = q0 * dy;
  M[2] += q2;
  const double q3 = q0 * dz;
  M[3] += q3;
  const double q4 = q1 * dx;
  M[4] += q4;
  const double q5 = q2 * dx;
  M[5] += q5;
  const double q6 = q3 * dx;
  M[6] += q6;
  const double q7 = q2 * dy;
  M[7] += q7;
  const double q8 = q3 * dy;
  M[8] += q8;
  const double q9 = q3 * dz;
  M[9] += q9;
}

__device__ __forceinline__ void m2m_acc_p2(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  const double w4 = w1 * sx;
  const double w5 = w2 * sx;
  const double w6 = w3 * sx;
  const double w7 = w2 * sy;
  const double w8 = w3 * sy;
  const double w9 = w3 * sz;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
  Mp[1] = fma(w0, Mc[1], fma(w1, Mc[0], Mp[1]));
  Mp[2] = fma(w0, Mc[2], fma(w2, Mc[0], Mp[2]));
  Mp[3] = fma(w0, Mc[3], fma(w3, Mc[0], Mp[3]));
  Mp[4] = fma(w0, Mc[4], fma(w1 * 2.0, Mc[1], fma(w4, Mc[0], Mp[4])));
  Mp[5] = fma(w0, Mc[5], fma(w2, Mc[1], fma(w1, Mc[2], fma(w5, Mc[0], Mp[5]))));
  Mp[6] = fma(w0, Mc[6], fma(w3, Mc[1], fma(w1, Mc[3], fma(w6, Mc[0], Mp[6]))));
  Mp[7] = fma(w0, Mc[7], fma(w2 * 2.0, Mc[2], fma(w7, Mc[0], Mp[7])));
  Mp[8] = fma(w0, Mc[8], fma(w3, Mc[2], fma(w2, Mc[3], fma(w8, Mc[0], Mp[8]))));
  Mp[9] = fma(w0, Mc[9], fma(w3 * 2.0, Mc[3], fma(w9, Mc[0], Mp[9])));
}

__device__ __forceinline__ void p2m_acc_p3(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
  const double q1 = q0 * dx;
  M[1] += q1;
  const double q2 = q0 * dy;
  M[2] += q2;
  const double q3 = q0 * dz;
  M[3] += q3;
  const double q4 = q1 * dx;
  M[4] += q4;
  const double q5 = q2 * dx;
  M[5] += q5;
  const double q6 = q3 * dx;
  M[6] += q6;
  const double q7 = q2 * dy;
  M[7] += q7;
  const double q8 = q3 * dy;
  M[8] += q8;
  const double q9 = q3 * dz;
  M[9] += q9;
  const double q10 = q4 * dx;
  M[10] += q10;
  const double q11 = q5 * dx;
  M[11] += q11;
  const double q12 = q6 * dx;
  M[12] += q12;
  const double q13 = q7 * dx;
  M[13] += q13;
  const double q14 = q8 * dx;
  M[14] += q14;
  const double q15 = q9 * dx;
  M[15] += q15;
  const double q16 = q7 * dy;
  M[16] += q16;
  const double q17 = q8 * dy;
  M[17] += q17;
  const double q18 = q9 * dy;
  M[18] += q18;
  const double q19 = q9 * dz;
  M[19] += q19;
}

__device__ __forceinline__ void m2m_acc_p3(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  const double w4 = w1 * sx;
  const double w5 = w2 * sx;
  const double w6 = w3 * sx;
  const double w7 = w2 * sy;
  const double w8 = w3 * sy;
  const double w9 = w3 * sz;
  const double w10 = w4 * sx;
  const double w11 = w5 * sx;
  const double w12 = w6 * sx;
  const double w13 = w7 * sx;
  const double w14 = w8 * sx;
  const double w15 = w9 * sx;
  const double w16 = w7 * sy;
  const double w17 = w8 * sy;
  const double w18 = w9 * sy;
  const double w19 = w9 * sz;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
  Mp[1] = fma(w0, Mc[1], fma(w1, Mc[0], Mp[1]));
  Mp[2] = fma(w0, Mc[2], fma(w2, Mc[0], Mp[2]));
  Mp[3] = fma(w0, Mc[3], fma(w3, Mc[0], Mp[3]));
  Mp[4] = fma(w0, Mc[4], fma(w1 * 2.0, Mc[1], fma(w4, Mc[0], Mp[4])));
  Mp[5] = fma(w0, Mc[5], fma(w2, Mc[1], fma(w1, Mc[2], fma(w5, Mc[0], Mp[5]))));
  Mp[6] = fma(w0, Mc[6], fma(w3, Mc[1], fma(w1, Mc[3], fma(w6, Mc[0], Mp[6]))));
  Mp[7] = fma(w0, Mc[7], fma(w2 * 2.0, Mc[2], fma(w7, Mc[0], Mp[7])));
  Mp[8] = fma(w0, Mc[8], fma(w3, Mc[2], fma(w2, Mc[3], fma(w8, Mc[0], Mp[8]))));
  Mp[9] = fma(w0, Mc[9], fma(w3 * 2.0, Mc[3], fma(w9, Mc[0], Mp[9])));
  Mp[10] = fma(w0, Mc[10], fma(w1 * 3.0, Mc[4], fma(w4 * 3.0, Mc[1], fma(w10, Mc[0], Mp[10]))));
  Mp[11] = fma(w0, Mc[11], fma(w2, Mc[4], fma(w1 * 2.0, Mc[5], fma(w5 * 2.0, Mc[1], fma(w4, Mc[2], fma(w11, Mc[0], Mp[11]))))));
  Mp[12] = fma(w0, Mc[12], fma(w3, Mc[4], fma(w1 * 2.0, Mc[6], fma(w6 * 2.0, Mc[1], fma(w4, Mc[3], fma(w12, Mc[0], Mp[12]))))));
  Mp[13] = fma(w0, Mc[13], fma(w2 * 2.0, Mc[5], fma(w7, Mc[1], fma(w1, Mc[7], fma(w5 * 2.0, Mc[2], fma(w13, Mc[0], Mp[13]))))));
  Mp[14] = fma(w0, Mc[14], fma(w3, Mc[5], fma(w2, Mc[6], fma(w8, Mc[1], fma(w1, Mc[8], fma(w6, Mc[2], fma(w5, Mc[3], fma(w14, Mc[0], Mp[14]))))))));
  Mp[15] = fma(w0, Mc[15], fma(w3 * 2.0, Mc[6], fma(w9, Mc[1], fma(w1, Mc[9], fma(w6 * 2.0, Mc[3], fma(w15, Mc[0], Mp[15]))))));
  Mp[16] = fma(w0, Mc[16], fma(w2 * 3.0, Mc[7], fma(w7 * 3.0, Mc[2], fma(w16, Mc[0], Mp[16]))));
  Mp[17] = fma(w0, Mc[17], fma(w3, Mc[7], fma(w2 * 2.0, Mc[8], fma(w8 * 2.0, Mc[2], fma(w7, Mc[3], fma(w17, Mc[0], Mp[17]))))));
  Mp[18] = fma(w0, Mc[18], fma(w3 * 2.0, Mc[8], fma(w9, Mc[2], fma(w2, Mc[9], fma(w8 * 2.0, Mc[3], fma(w18, Mc[0], Mp[18]))))));
  Mp[19] = fma(w0, Mc[19], fma(w3 * 3.0, Mc[9], fma(w9 * 3.0, Mc[3], fma(w19, Mc[0], Mp[19]))));
}

__device__ __forceinline__ void p2m_acc_p4(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
  const double q1 = q0 * dx;
  M[1] += q1;
  const double q2 = q0 * dy;
  M[2] += q2;
  const double q3 = q0 * dz;
  M[3] += q3;
  const double q4 = q1 * dx;
  M[4] += q4;
  const double q5 = q2 * dx;
  M[5] += q5;
  const double q6 = q3 * dx;
  M[6] += q6;
  const double q7 = q2 * dy;
  M[7] += q7;
  const double q8 = q3 * dy;
  M[8] += q8;
  const double q9 = q3 * dz;
  M[9] += q9;
  const double q10 = q4 * dx;
  M[10] += q10;
  const double q11 = q5 * dx;
  M[11] += q11;
  const double q12 = q6 * dx;
  M[12] += q12;
  const double q13 = q7 * dx;
  M[13] += q13;
  const double q14 = q8 * dx;
  M[14] += q14;
  const double q15 = q9 * dx;
  M[15] += q15;
  const double q16 = q7 * dy;
  M[16] += q16;
  const double q17 = q8 * dy;
  M[17] += q17;
  const double q18 = q9 * dy;
  M[18] += q18;
  const double q19 = q9 * dz;
  M[19] += q19;
  const double q20 = q10 * dx;
  M[20] += q20;
  const double q21 = q11 * dx;
  M[21] += q21;
  const double q22 = q12 * dx;
  M[22] += q22;
  const double q23 = q13 * dx;
  M[23] += q23;
  const double q24 = q14 * dx;
  M[24] += q24;
  const double q25 = q15 * dx;
  M[25] += q25;
  const double q26 = q16 * dx;
  M[26] += q26;
  const double q27 = q17 * dx;
  M[27] += q27;
  const double q28 = q18 * dx;
  M[28] += q28;
  const double q29 = q19 * dx;
  M[29] += q29;
  const double q30 = q16 * dy;
  M[30] += q30;
  const double q31 = q17 * dy;
  M[31] += q31;
  const double q32 = q18 * dy;
  M[32] += q32;
  const double q33 = q19 * dy;
  M[33] += q33;
  const double q34 = q19 * dz;
  M[34] += q34;
}

__device__ __forceinline__ void m2m_acc_p4(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  const double w4 = w1 * sx;
  const double w5 = w2 * sx;
  const double w6 = w3 * sx;
  const double w7 = w2 * sy;
  const double w8 = w3 * sy;
  const double w9 = w3 * sz;
  const double w10 = w4 * sx;
  const double w11 = w5 * sx;
  const double w12 = w6 * sx;
  const double w13 = w7 * sx;
  const double w14 = w8 * sx;
  const double w15 = w9 * sx;
  const double w16 = w7 * sy;
  const double w17 = w8 * sy;
  const double w18 = w9 * sy;
  const double w19 = w9 * sz;
  const double w20 = w10 * sx;
  const double w21 = w11 * sx;
  const double w22 = w12 * sx;
  const double w23 = w13 * sx;
  const double w24 = w14 * sx;
  const double w25 = w15 * sx;
  const double w26 = w16 * sx;
  const double w27 = w17 * sx;
  const double w28 = w18 * sx;
  const double w29 = w19 * sx;
  const double w30 = w16 * sy;
  const double w31 = w17 * sy;
  const double w32 = w18 * sy;
  const double w33 = w19 * sy;
  const double w34 = w19 * sz;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
  Mp[1] = fma(w0, Mc[1], fma(w1, Mc[0], Mp[1]));
  Mp[2] = fma(w0, Mc[2], fma(w2, Mc[0], Mp[2]));
  Mp[3] = fma(w0, Mc[3], fma(w3, Mc[0], Mp[3]));
  Mp[4] = fma(w0, Mc[4], fma(w1 * 2.0, Mc[1], fma(w4, Mc[0], Mp[4])));
  Mp[5] = fma(w0, Mc[5], fma(w2, Mc[1], fma(w1, Mc[2], fma(w5, Mc[0], Mp[5]))));
  Mp[6] = fma(w0, Mc[6], fma(w3, Mc[1], fma(w1, Mc[3], fma(w6, Mc[0], Mp[6]))));
  Mp[7] = fma(w0, Mc[7], fma(w2 * 2.0, Mc[2], fma(w7, Mc[0], Mp[7])));
  Mp[8] = fma(w0, Mc[8], fma(w3, Mc[2], fma(w2, Mc[3], fma(w8, Mc[0], Mp[8]))));
  Mp[9] = fma(w0, Mc[9], fma(w3 * 2.0, Mc[3], fma(w9, Mc[0], Mp[9])));
  Mp[10] = fma(w0, Mc[10], fma(w1 * 3.0, Mc[4], fma(w4 * 3.0, Mc[1], fma(w10, Mc[0], Mp[10]))));
  Mp[11] = fma(w0, Mc[11], fma(w2, Mc[4], fma(w1 * 2.0, Mc[5], fma(w5 * 2.0, Mc[1], fma(w4, Mc[2], fma(w11, Mc[0], Mp[11]))))));
  Mp[12] = fma(w0, Mc[12], fma(w3, Mc[4], fma(w1 * 2.0, Mc[6], fma(w6 * 2.0, Mc[1], fma(w4, Mc[3], fma(w12, Mc[0], Mp[12]))))));
  Mp[13] = fma(w0, Mc[13], fma(w2 * 2.0, Mc[5], fma(w7, Mc[1], fma(w1, Mc[7], fma(w5 * 2.0, Mc[2], fma(w13, Mc[0], Mp[13]))))));
  Mp[14] = fma(w0, Mc[14], fma(w3, Mc[5], fma(w2, Mc[6], fma(w8, Mc[1], fma(w1, Mc[8], fma(w6, Mc[2], fma(w5, Mc[3], fma(w14, Mc[0], Mp[14]))))))));
  Mp[15] = fma(w0, Mc[15], fma(w3 * 2.0, Mc[6], fma(w9, Mc[1], fma(w1, Mc[9], fma(w6 * 2.0, Mc[3], fma(w15, Mc[0], Mp[15]))))));
  Mp[16] = fma(w0, Mc[16], fma(w2 * 3.0, Mc[7], fma(w7 * 3.0, Mc[2], fma(w16, Mc[0], Mp[16]))));
  Mp[17] = fma(w0, Mc[17], fma(w3, Mc[7], fma(w2 * 2.0, Mc[8], fma(w8 * 2.0, Mc[2], fma(w7, Mc[3], fma(w17, Mc[0], Mp[17]))))));
  Mp[18] = fma(w0, Mc[18], fma(w3 * 2.0, Mc[8], fma(w9, Mc[2], fma(w2, Mc[9], fma(w8 * 2.0, Mc[3], fma(w18, Mc[0], Mp[18]))))));
  Mp[19] = fma(w0, Mc[19], fma(w3 * 3.0, Mc[9], fma(w9 * 3.0, Mc[3], fma(w19, Mc[0], Mp[19]))));
  Mp[20] = fma(w0, Mc[20], fma(w1 * 4.0, Mc[10], fma(w4 * 6.0, Mc[4], fma(w10 * 4.0, Mc[1], fma(w20, Mc[0], Mp[20])))));
  Mp[21] = fma(w0, Mc[21], fma(w2, Mc[10], fma(w1 * 3.0, Mc[11], fma(w5 * 3.0, Mc[4], fma(w4 * 3.0, Mc[5], fma(w11 * 3.0, Mc[1], fma(w10, Mc[2], fma(w21, Mc[0], Mp[21]))))))));
  Mp[22] = fma(w0, Mc[22], fma(w3, Mc[10], fma(w1 * 3.0, Mc[12], fma(w6 * 3.0, Mc[4], fma(w4 * 3.0, Mc[6], fma(w12 * 3.0, Mc[1], fma(w10, Mc[3], fma(w22, Mc[0], Mp[22]))))))));
  Mp[23] = fma(w0, Mc[23], fma(w2 * 2.0, Mc[11], fma(w7, Mc[4], fma(w1 * 2.0, Mc[13], fma(w5 * 4.0, Mc[5], fma(w13 * 2.0, Mc[1], fma(w4, Mc[7], fma(w11 * 2.0, Mc[2], fma(w23, Mc[0], Mp[23])))))))));
  Mp[24] = fma(w0, Mc[24], fma(w3, Mc[11], fma(w2, Mc[12], fma(w8, Mc[4], fma(w1 * 2.0, Mc[14], fma(w6 * 2.0, Mc[5], fma(w5 * 2.0, Mc[6], fma(w14 * 2.0, Mc[1], fma(w4, Mc[8], fma(w12, Mc[2], fma(w11, Mc[3], fma(w24, Mc[0], Mp[24]))))))))))));
  Mp[25] = fma(w0, Mc[25], fma(w3 * 2.0, Mc[12], fma(w9, Mc[4], fma(w1 * 2.0, Mc[15], fma(w6 * 4.0, Mc[6], fma(w15 * 2.0, Mc[1], fma(w4, Mc[9], fma(w12 * 2.0, Mc[3], fma(w25, Mc[0], Mp[25])))))))));
  Mp[26] = fma(w0, Mc[26], fma(w2 * 3.0, Mc[13], fma(w7 * 3.0, Mc[5], fma(w16, Mc[1], fma(w1, Mc[16], fma(w5 * 3.0, Mc[7], fma(w13 * 3.0, Mc[2], fma(w26, Mc[0], Mp[26]))))))));
  Mp[27] = fma(w0, Mc[27], fma(w3, Mc[13], fma(w2 * 2.0, Mc[14], fma(w8 * 2.0, Mc[5], fma(w7, Mc[6], fma(w17, Mc[1], fma(w1, Mc[17], fma(w6, Mc[7], fma(w5 * 2.0, Mc[8], fma(w14 * 2.0, Mc[2], fma(w13, Mc[3], fma(w27, Mc[0], Mp[27]))))))))))));
  Mp[28] = fma(w0, Mc[28], fma(w3 * 2.0, Mc[14], fma(w9, Mc[5], fma(w2, Mc[15], fma(w8 * 2.0, Mc[6], fma(w18, Mc[1], fma(w1, Mc[18], fma(w6 * 2.0, Mc[8], fma(w15, Mc[2], fma(w5, Mc[9], fma(w14 * 2.0, Mc[3], fma(w28, Mc[0], Mp[28]))))))))))));
  Mp[29] = fma(w0, Mc[29], fma(w3 * 3.0, Mc[15], fma(w9 * 3.0, Mc[6], fma(w19, Mc[1], fma(w1, Mc[19], fma(w6 * 3.0, Mc[9], fma(w15 * 3.0, Mc[3], fma(w29, Mc[0], Mp[29]))))))));
  Mp[30] = fma(w0, Mc[30], fma(w2 * 4.0, Mc[16], fma(w7 * 6.0, Mc[7], fma(w16 * 4.0, Mc[2], fma(w30, Mc[0], Mp[30])))));
  Mp[31] = fma(w0, Mc[31], fma(w3, Mc[16], fma(w2 * 3.0, Mc[17], fma(w8 * 3.0, Mc[7], fma(w7 * 3.0, Mc[8], fma(w17 * 3.0, Mc[2], fma(w16, Mc[3], fma(w31, Mc[0], Mp[31]))))))));
  Mp[32] = fma(w0, Mc[32], fma(w3 * 2.0, Mc[17], fma(w9, Mc[7], fma(w2 * 2.0, Mc[18], fma(w8 * 4.0, Mc[8], fma(w18 * 2.0, Mc[2], fma(w7, Mc[9], fma(w17 * 2.0, Mc[3], fma(w32, Mc[0], Mp[32])))))))));
  Mp[33] = fma(w0, Mc[33], fma(w3 * 3.0, Mc[18], fma(w9 * 3.0, Mc[8], fma(w19, Mc[2], fma(w2, Mc[19], fma(w8 * 3.0, Mc[9], fma(w18 * 3.0, Mc[3], fma(w33, Mc[0], Mp[33]))))))));
  Mp[34] = fma(w0, Mc[34], fma(w3 * 4.0, Mc[19], fma(w9 * 6.0, Mc[9], fma(w19 * 4.0, Mc[3], fma(w34, Mc[0], Mp[34])))));
}

__device__ __forceinline__ void p2m_acc_p5(double m, double dx, double dy, double dz, double* __restrict__ M) {
  const double q0 = m;
  M[0] += q0;
  const double q1 = q0 * dx;
  M[1] += q1;
  const double q2 = q0 * dy;
  M[2] += q2;
  const double q3 = q0 * dz;
  M[3] += q3;
  const double q4 = q1 * dx;
  M[4] += q4;
  const double q5 = q2 * dx;
  M[5] += q5;
  const double q6 = q3 * dx;
  M[6] += q6;
  const double q7 = q2 * dy;
  M[7] += q7;
  const double q8 = q3 * dy;
  M[8] += q8;
  const double q9 = q3 * dz;
  M[9] += q9;
  const double q10 = q4 * dx;
  M[10] += q10;
  const double q11 = q5 * dx;
  M[11] += q11;
  const double q12 = q6 * dx;
  M[12] += q12;
  const double q13 = q7 * dx;
  M[13] += q13;
  const double q14 = q8 * dx;
  M[14] += q14;
  const double q15 = q9 * dx;
  M[15] += q15;
  const double q16 = q7 * dy;
  M[16] += q16;
  const double q17 = q8 * dy;
  M[17] += q17;
  const double q18 = q9 * dy;
  M[18] += q18;
  const double q19 = q9 * dz;
  M[19] += q19;
  const double q20 = q10 * dx;
  M[20] += q20;
  const double q21 = q11 * dx;
  M[21] += q21;
  const double q22 = q12 * dx;
  M[22] += q22;
  const double q23 = q13 * dx;
  M[23] += q23;
  const double q24 = q14 * dx;
  M[24] += q24;
  const double q25 = q15 * dx;
  M[25] += q25;
  const double q26 = q16 * dx;
  M[26] += q26;
  const double q27 = q17 * dx;
  M[27] += q27;
  const double q28 = q18 * dx;
  M[28] += q28;
  const double q29 = q19 * dx;
  M[29] += q29;
  const double q30 = q16 * dy;
  M[30] += q30;
  const double q31 = q17 * dy;
  M[31] += q31;
  const double q32 = q18 * dy;
  M[32] += q32;
  const double q33 = q19 * dy;
  M[33] += q33;
  const double q34 = q19 * dz;
  M[34] += q34;
  const double q35 = q20 * dx;
  M[35] += q35;
  const double q36 = q21 * dx;
  M[36] += q36;
  const double q37 = q22 * dx;
  M[37] += q37;
  const double q38 = q23 * dx;
  M[38] += q38;
  const double q39 = q24 * dx;
  M[39] += q39;
  const double q40 = q25 * dx;
  M[40] += q40;
  const double q41 = q26 * dx;
  M[41] += q41;
  const double q42 = q27 * dx;
  M[42] += q42;
  const double q43 = q28 * dx;
  M[43] += q43;
  const double q44 = q29 * dx;
  M[44] += q44;
  const double q45 = q30 * dx;
  M[45] += q45;
  const double q46 = q31 * dx;
  M[46] += q46;
  const double q47 = q32 * dx;
  M[47] += q47;
  const double q48 = q33 * dx;
  M[48] += q48;
  const double q49 = q34 * dx;
  M[49] += q49;
  const double q50 = q30 * dy;
  M[50] += q50;
  const double q51 = q31 * dy;
  M[51] += q51;
  const double q52 = q32 * dy;
  M[52] += q52;
  const double q53 = q33 * dy;
  M[53] += q53;
  const double q54 = q34 * dy;
  M[54] += q54;
  const double q55 = q34 * dz;
  M[55] += q55;
}

__device__ __forceinline__ void m2m_acc_p5(const double* __restrict__ Mc, double sx, double sy, double sz, double* __restrict__ Mp) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  const double w4 = w1 * sx;
  const double w5 = w2 * sx;
  const double w6 = w3 * sx;
  const double w7 = w2 * sy;
  const double w8 = w3 * sy;
  const double w9 = w3 * sz;
  const double w10 = w4 * sx;
  const double w11 = w5 * sx;
  const double w12 = w6 * sx;
  const double w13 = w7 * sx;
  const double w14 = w8 * sx;
  const double w15 = w9 * sx;
  const double w16 = w7 * sy;
  const double w17 = w8 * sy;
  const double w18 = w9 * sy;
  const double w19 = w9 * sz;
  const double w20 = w10 * sx;
  const double w21 = w11 * sx;
  const double w22 = w12 * sx;
  const double w23 = w13 * sx;
  const double w24 = w14 * sx;
  const double w25 = w15 * sx;
  const double w26 = w16 * sx;
  const double w27 = w17 * sx;
  const double w28 = w18 * sx;
  const double w29 = w19 * sx;
  const double w30 = w16 * sy;
  const double w31 = w17 * sy;
  const double w32 = w18 * sy;
  const double w33 = w19 * sy;
  const double w34 = w19 * sz;
  const double w35 = w20 * sx;
  const double w36 = w21 * sx;
  const double w37 = w22 * sx;
  const double w38 = w23 * sx;
  const double w39 = w24 * sx;
  const double w40 = w25 * sx;
  const double w41 = w26 * sx;
  const double w42 = w27 * sx;
  const double w43 = w28 * sx;
  const double w44 = w29 * sx;
  const double w45 = w30 * sx;
  const double w46 = w31 * sx;
  const double w47 = w32 * sx;
  const double w48 = w33 * sx;
  const double w49 = w34 * sx;
  const double w50 = w30 * sy;
  const double w51 = w31 * sy;
  const double w52 = w32 * sy;
  const double w53 = w33 * sy;
  const double w54 = w34 * sy;
  const double w55 = w34 * sz;
  Mp[0] = fma(w0, Mc[0], Mp[0]);
  Mp[1] = fma(w0, Mc[1], fma(w1, Mc[0], Mp[1]));
  Mp[2] = fma(w0, Mc[2], fma(w2, Mc[0], Mp[2]));
  Mp[3] = fma(w0, Mc[3], fma(w3, Mc[0], Mp[3]));
  Mp[4] = fma(w0, Mc[4], fma(w1 * 2.0, Mc[1], fma(w4, Mc[0], Mp[4])));
  Mp[5] = fma(w0, Mc[5], fma(w2, Mc[1], fma(w1, Mc[2], fma(w5, Mc[0], Mp[5]))));
  Mp[6] = fma(w0, Mc[6], fma(w3, Mc[1], fma(w1, Mc[3], fma(w6, Mc[0], Mp[6]))));
  Mp[7] = fma(w0, Mc[7], fma(w2 * 2.0, Mc[2], fma(w7, Mc[0], Mp[7])));
  Mp[8] = fma(w0, Mc[8], fma(w3, Mc[2], fma(w2, Mc[3], fma(w8, Mc[0], Mp[8]))));
  Mp[9] = fma(w0, Mc[9], fma(w3 * 2.0, Mc[3], fma(w9, Mc[0], Mp[9])));
  Mp[10] = fma(w0, Mc[10], fma(w1 * 3.0, Mc[4], fma(w4 * 3.0, Mc[1], fma(w10, Mc[0], Mp[10]))));
  Mp[11] = fma(w0, Mc[11], fma(w2, Mc[4], fma(w1 * 2.0, Mc[5], fma(w5 * 2.0, Mc[1], fma(w4, Mc[2], fma(w11, Mc[0], Mp[11]))))));
  Mp[12] = fma(w0, Mc[12], fma(w3, Mc[4], fma(w1 * 2.0, Mc[6], fma(w6 * 2.0, Mc[1], fma(w4, Mc[3], fma(w12, Mc[0], Mp[12]))))));
  Mp[13] = fma(w0, Mc[13], fma(w2 * 2.0, Mc[5], fma(w7, Mc[1], fma(w1, Mc[7], fma(w5 * 2.0, Mc[2], fma(w13, Mc[0], Mp[13]))))));
  Mp[14] = fma(w0, Mc[14], fma(w3, Mc[5], fma(w2, Mc[6], fma(w8, Mc[1], fma(w1, Mc[8], fma(w6, Mc[2], fma(w5, Mc[3], fma(w14, Mc[0], Mp[14]))))))));
  Mp[15] = fma(w0, Mc[15], fma(w3 * 2.0, Mc[6], fma(w9, Mc[1], fma(w1, Mc[9], fma(w6 * 2.0, Mc[3], fma(w15, Mc[0], Mp[15]))))));
  Mp[16] = fma(w0, Mc[16], fma(w2 * 3.0, Mc[7], fma(w7 * 3.0, Mc[2], fma(w16, Mc[0], Mp[16]))));
  Mp[17] = fma(w0, Mc[17], fma(w3, Mc[7], fma(w2 * 2.0, Mc[8], fma(w8 * 2.0, Mc[2], fma(w7, Mc[3], fma(w17, Mc[0], Mp[17]))))));
  Mp[18] = fma(w0, Mc[18], fma(w3 * 2.0, Mc[8], fma(w9, Mc[2], fma(w2, Mc[9], fma(w8 * 2.0, Mc[3], fma(w18, Mc[0], Mp[18]))))));
  Mp[19] = fma(w0, Mc[19], fma(w3 * 3.0, Mc[9], fma(w9 * 3.0, Mc[3], fma(w19, Mc[0], Mp[19]))));
  Mp[20] = fma(w0, Mc[20], fma(w1 * 4.0, Mc[10], fma(w4 * 6.0, Mc[4], fma(w10 * 4.0, Mc[1], fma(w20, Mc[0], Mp[20])))));
  Mp[21] = fma(w0, Mc[21], fma(w2, Mc[10], fma(w1 * 3.0, Mc[11], fma(w5 * 3.0, Mc[4], fma(w4 * 3.0, Mc[5], fma(w11 * 3.0, Mc[1], fma(w10, Mc[2], fma(w21, Mc[0], Mp[21]))))))));
  Mp[22] = fma(w0, Mc[22], fma(w3, Mc[10], fma(w1 * 3.0, Mc[12], fma(w6 * 3.0, Mc[4], fma(w4 * 3.0, Mc[6], fma(w12 * 3.0, Mc[1], fma(w10, Mc[3], fma(w22, Mc[0], Mp[22]))))))));
  Mp[23] = fma(w0, Mc[23], fma(w2 * 2.0, Mc[11], fma(w7, Mc[4], fma(w1 * 2.0, Mc[13], fma(w5 * 4.0, Mc[5], fma(w13 * 2.0, Mc[1], fma(w4, Mc[7], fma(w11 * 2.0, Mc[2], fma(w23, Mc[0], Mp[23])))))))));
  Mp[24] = fma(w0, Mc[24], fma(w3, Mc[11], fma(w2, Mc[12], fma(w8, Mc[4], fma(w1 * 2.0, Mc[14], fma(w6 * 2.0, Mc[5], fma(w5 * 2.0, Mc[6], fma(w14 * 2.0, Mc[1], fma(w4, Mc[8], fma(w12, Mc[2], fma(w11, Mc[3], fma(w24, Mc[0], Mp[24]))))))))))));
  Mp[25] = fma(w0, Mc[25], fma(w3 * 2.0, Mc[12], fma(w9, Mc[4], fma(w1 * 2.0, Mc[15], fma(w6 * 4.0, Mc[6], fma(w15 * 2.0, Mc[1], fma(w4, Mc[9], fma(w12 * 2.0, Mc[3], fma(w25, Mc[0], Mp[25])))))))));
  Mp[26] = fma(w0, Mc[26], fma(w2 * 3.0, Mc[13], fma(w7 * 3.0, Mc[5], fma(w16, Mc[1], fma(w1, Mc[16], fma(w5 * 3.0, Mc[7], fma(w13 * 3.0, Mc[2], fma(w26, Mc[0], Mp[26]))))))));
  Mp[27] = fma(w0, Mc[27], fma(w3, Mc[13], fma(w2 * 2.0, Mc[14], fma(w8 * 2.0, Mc[5], fma(w7, Mc[6], fma(w17, Mc[1], fma(w1, Mc[17], fma(w6, Mc[7], fma(w5 * 2.0, Mc[8], fma(w14 * 2.0, Mc[2], fma(w13, Mc[3], fma(w27, Mc[0], Mp[27]))))))))))));
  Mp[28] = fma(w0, Mc[28], fma(w3 * 2.0, Mc[14], fma(w9, Mc[5], fma(w2, Mc[15], fma(w8 * 2.0, Mc[6], fma(w18, Mc[1], fma(w1, Mc[18], fma(w6 * 2.0, Mc[8], fma(w15, Mc[2], fma(w5, Mc[9], fma(w14 * 2.0, Mc[3], fma(w28, Mc[0], Mp[28]))))))))))));
  Mp[29] = fma(w0, Mc[29], fma(w3 * 3.0, Mc[15], fma(w9 * 3.0, Mc[6], fma(w19, Mc[1], fma(w1, Mc[19], fma(w6 * 3.0, Mc[9], fma(w15 * 3.0, Mc[3], fma(w29, Mc[0], Mp[29]))))))));
  Mp[30] = fma(w0, Mc[30], fma(w2 * 4.0, Mc[16], fma(w7 * 6.0, Mc[7], fma(w16 * 4.0, Mc[2], fma(w30, Mc[0], Mp[30])))));
  Mp[31] = fma(w0, Mc[31], fma(w3, Mc[16], fma(w2 * 3.0, Mc[17], fma(w8 * 3.0, Mc[7], fma(w7 * 3.0, Mc[8], fma(w17 * 3.0, Mc[2], fma(w16, Mc[3], fma(w31, Mc[0], Mp[31]))))))));
  Mp[32] = fma(w0, Mc[32], fma(w3 * 2.0, Mc[17], fma(w9, Mc[7], fma(w2 * 2.0, Mc[18], fma(w8 * 4.0, Mc[8], fma(w18 * 2.0, Mc[2], fma(w7, Mc[9], fma(w17 * 2.0, Mc[3], fma(w32, Mc[0], Mp[32])))))))));
  Mp[33] = fma(w0, Mc[33], fma(w3 * 3.0, Mc[18], fma(w9 * 3.0, Mc[8], fma(w19, Mc[2], fma(w2, Mc[19], fma(w8 * 3.0, Mc[9], fma(w18 * 3.0, Mc[3], fma(w33, Mc[0], Mp[33]))))))));
  Mp[34] = fma(w0, Mc[34], fma(w3 * 4.0, Mc[19], fma(w9 * 6.0, Mc[9], fma(w19 * 4.0, Mc[3], fma(w34, Mc[0], Mp[34])))));
  Mp[35] = fma(w0, Mc[35], fma(w1 * 5.0, Mc[20], fma(w4 * 10.0, Mc[10], fma(w10 * 10.0, Mc[4], fma(w20 * 5.0, Mc[1], fma(w35, Mc[0], Mp[35]))))));
  Mp[36] = fma(w0, Mc[36], fma(w2, Mc[20], fma(w1 * 4.0, Mc[21], fma(w5 * 4.0, Mc[10], fma(w4 * 6.0, Mc[11], fma(w11 * 6.0, Mc[4], fma(w10 * 4.0, Mc[5], fma(w21 * 4.0, Mc[1], fma(w20, Mc[2], fma(w36, Mc[0], Mp[36]))))))))));
  Mp[37] = fma(w0, Mc[37], fma(w3, Mc[20], fma(w1 * 4.0, Mc[22], fma(w6 * 4.0, Mc[10], fma(w4 * 6.0, Mc[12], fma(w12 * 6.0, Mc[4], fma(w10 * 4.0, Mc[6], fma(w22 * 4.0, Mc[1], fma(w20, Mc[3], fma(w37, Mc[0], Mp[37]))))))))));
  Mp[38] = fma(w0, Mc[38], fma(w2 * 2.0, Mc[21], fma(w7, Mc[10], fma(w1 * 3.0, Mc[23], fma(w5 * 6.0, Mc[11], fma(w13 * 3.0, Mc[4], fma(w4 * 3.0, Mc[13], fma(w11 * 6.0, Mc[5], fma(w23 * 3.0, Mc[1], fma(w10, Mc[7], fma(w21 * 2.0, Mc[2], fma(w38, Mc[0], Mp[38]))))))))))));
  Mp[39] = fma(w0, Mc[39], fma(w3, Mc[21], fma(w2, Mc[22], fma(w8, Mc[10], fma(w1 * 3.0, Mc[24], fma(w6 * 3.0, Mc[11], fma(w5 * 3.0, Mc[12], fma(w14 * 3.0, Mc[4], fma(w4 * 3.0, Mc[14], fma(w12 * 3.0, Mc[5], fma(w11 * 3.0, Mc[6], fma(w24 * 3.0, Mc[1], fma(w10, Mc[8], fma(w22, Mc[2], fma(w21, Mc[3], fma(w39, Mc[0], Mp[39]))))))))))))))));
  Mp[40] = fma(w0, Mc[40], fma(w3 * 2.0, Mc[22], fma(w9, Mc[10], fma(w1 * 3.0, Mc[25], fma(w6 * 6.0, Mc[12], fma(w15 * 3.0, Mc[4], fma(w4 * 3.0, Mc[15], fma(w12 * 6.0, Mc[6], fma(w25 * 3.0, Mc[1], fma(w10, Mc[9], fma(w22 * 2.0, Mc[3], fma(w40, Mc[0], Mp[40]))))))))))));
  Mp[41] = fma(w0, Mc[41], fma(w2 * 3.0, Mc[23], fma(w7 * 3.0, Mc[11], fma(w16, Mc[4], fma(w1 * 2.0, Mc[26], fma(w5 * 6.0, Mc[13], fma(w13 * 6.0, Mc[5], fma(w26 * 2.0, Mc[1], fma(w4, Mc[16], fma(w11 * 3.0, Mc[7], fma(w23 * 3.0, Mc[2], fma(w41, Mc[0], Mp[41]))))))))))));
  Mp[42] = fma(w0, Mc[42], fma(w3, Mc[23], fma(w2 * 2.0, Mc[24], fma(w8 * 2.0, Mc[11], fma(w7, Mc[12], fma(w17, Mc[4], fma(w1 * 2.0, Mc[27], fma(w6 * 2.0, Mc[13], fma(w5 * 4.0, Mc[14], fma(w14 * 4.0, Mc[5], fma(w13 * 2.0, Mc[6], fma(w27 * 2.0, Mc[1], fma(w4, Mc[17], fma(w12, Mc[7], fma(w11 * 2.0, Mc[8], fma(w24 * 2.0, Mc[2], fma(w23, Mc[3], fma(w42, Mc[0], Mp[42]))))))))))))))))));
  Mp[43] = fma(w0, Mc[43], fma(w3 * 2.0, Mc[24], fma(w9, Mc[11], fma(w2, Mc[25], fma(w8 * 2.0, Mc[12], fma(w18, Mc[4], fma(w1 * 2.0, Mc[28], fma(w6 * 4.0, Mc[14], fma(w15 * 2.0, Mc[5], fma(w5 * 2.0, Mc[15], fma(w14 * 4.0, Mc[6], fma(w28 * 2.0, Mc[1], fma(w4, Mc[18], fma(w12 * 2.0, Mc[8], fma(w25, Mc[2], fma(w11, Mc[9], fma(w24 * 2.0, Mc[3], fma(w43, Mc[0], Mp[43]))))))))))))))))));
  Mp[44] = fma(w0, Mc[44], fma(w3 * 3.0, Mc[25], fma(w9 * 3.0, Mc[12], fma(w19, Mc[4], fma(w1 * 2.0, Mc[29], fma(w6 * 6.0, Mc[15], fma(w15 * 6.0, Mc[6], fma(w29 * 2.0, Mc[1], fma(w4, Mc[19], fma(w12 * 3.0, Mc[9], fma(w25 * 3.0, Mc[3], fma(w44, Mc[0], Mp[44]))))))))))));
  Mp[45] = fma(w0, Mc[45], fma(w2 * 4.0, Mc[26], fma(w7 * 6.0, Mc[13], fma(w16 * 4.0, Mc[5], fma(w30, Mc[1], fma(w1, Mc[30], fma(w5 * 4.0, Mc[16], fma(w13 * 6.0, Mc[7], fma(w26 * 4.0, Mc[2], fma(w45, Mc[0], Mp[45]))))))))));
  Mp[46] = fma(w0, Mc[46], fma(w3, Mc[26], fma(w2 * 3.0, Mc[27], fma(w8 * 3.0, Mc[13], fma(w7 * 3.0, Mc[14], fma(w17 * 3.0, Mc[5], fma(w16, Mc[6], fma(w31, Mc[1], fma(w1, Mc[31], fma(w6, Mc[16], fma(w5 * 3.0, Mc[17], fma(w14 * 3.0, Mc[7], fma(w13 * 3.0, Mc[8], fma(w27 * 3.0, Mc[2], fma(w26, Mc[3], fma(w46, Mc[0], Mp[46]))))))))))))))));
  Mp[47] = fma(w0, Mc[47], fma(w3 * 2.0, Mc[27], fma(w9, Mc[13], fma(w2 * 2.0, Mc[28], fma(w8 * 4.0, Mc[14], fma(w18 * 2.0, Mc[5], fma(w7, Mc[15], fma(w17 * 2.0, Mc[6], fma(w32, Mc[1], fma(w1, Mc[32], fma(w6 * 2.0, Mc[17], fma(w15, Mc[7], fma(w5 * 2.0, Mc[18], fma(w14 * 4.0, Mc[8], fma(w28 * 2.0, Mc[2], fma(w13, Mc[9], fma(w27 * 2.0, Mc[3], fma(w47, Mc[0], Mp[47]))))))))))))))))));
  Mp[48] = fma(w0, Mc[48], fma(w3 * 3.0, Mc[28], fma(w9 * 3.0, Mc[14], fma(w19, Mc[5], fma(w2, Mc[29], fma(w8 * 3.0, Mc[15], fma(w18 * 3.0, Mc[6], fma(w33, Mc[1], fma(w1, Mc[33], fma(w6 * 3.0, Mc[18], fma(w15 * 3.0, Mc[8], fma(w29, Mc[2], fma(w5, Mc[19], fma(w14 * 3.0, Mc[9], fma(w28 * 3.0, Mc[3], fma(w48, Mc[0], Mp[48]))))))))))))))));
  Mp[49] = fma(w0, Mc[49], fma(w3 * 4.0, Mc[29], fma(w9 * 6.0, Mc[15], fma(w19 * 4.0, Mc[6], fma(w34, Mc[1], fma(w1, Mc[34], fma(w6 * 4.0, Mc[19], fma(w15 * 6.0, Mc[9], fma(w29 * 4.0, Mc[3], fma(w49, Mc[0], Mp[49]))))))))));
  Mp[50] = fma(w0, Mc[50], fma(w2 * 5.0, Mc[30], fma(w7 * 10.0, Mc[16], fma(w16 * 10.0, Mc[7], fma(w30 * 5.0, Mc[2], fma(w50, Mc[0], Mp[50]))))));
  Mp[51] = fma(w0, Mc[51], fma(w3, Mc[30], fma(w2 * 4.0, Mc[31], fma(w8 * 4.0, Mc[16], fma(w7 * 6.0, Mc[17], fma(w17 * 6.0, Mc[7], fma(w16 * 4.0, Mc[8], fma(w31 * 4.0, Mc[2], fma(w30, Mc[3], fma(w51, Mc[0], Mp[51]))))))))));
  Mp[52] = fma(w0, Mc[52], fma(w3 * 2.0, Mc[31], fma(w9, Mc[16], fma(w2 * 3.0, Mc[32], fma(w8 * 6.0, Mc[17], fma(w18 * 3.0, Mc[7], fma(w7 * 3.0, Mc[18], fma(w17 * 6.0, Mc[8], fma(w32 * 3.0, Mc[2], fma(w16, Mc[9], fma(w31 * 2.0, Mc[3], fma(w52, Mc[0], Mp[52]))))))))))));
  Mp[53] = fma(w0, Mc[53], fma(w3 * 3.0, Mc[32], fma(w9 * 3.0, Mc[17], fma(w19, Mc[7], fma(w2 * 2.0, Mc[33], fma(w8 * 6.0, Mc[18], fma(w18 * 6.0, Mc[8], fma(w33 * 2.0, Mc[2], fma(w7, Mc[19], fma(w17 * 3.0, Mc[9], fma(w32 * 3.0, Mc[3], fma(w53, Mc[0], Mp[53]))))))))))));
  Mp[54] = fma(w0, Mc[54], fma(w3 * 4.0, Mc[33], fma(w9 * 6.0, Mc[18], fma(w19 * 4.0, Mc[8], fma(w34, Mc[2], fma(w2, Mc[34], fma(w8 * 4.0, Mc[19], fma(w18 * 6.0, Mc[9], fma(w33 * 4.0, Mc[3], fma(w54, Mc[0], Mp[54]))))))))));
  Mp[55] = fma(w0, Mc[55], fma(w3 * 5.0, Mc[34], fma(w9 * 10.0, Mc[19], fma(w19 * 10.0, Mc[9], fma(w34 * 5.0, Mc[3], fma(w55, Mc[0], Mp[55]))))));
}

constexpr int kNL1 = 9;  // local coefficients, image-field order 1
template <typename T>
__device__ __forceinline__ void m2l_pe1(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {
  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..2)
  Lc[0] = fma(-M[3], D[6], fma(-M[2], D[5], fma(-M[1], D[4], fma(M[0], D[1], Lc[0]))));
  Lc[1] = fma(-M[3], D[8], fma(-M[2], D[7], fma(-M[1], D[5], fma(M[0], D[2], Lc[1]))));
  Lc[2] = fma(-M[3], D[9], fma(-M[2], D[8], fma(-M[1], D[6], fma(M[0], D[3], Lc[2]))));
  Lc[3] = fma(M[0], D[4], Lc[3]);
  Lc[4] = fma(M[0], D[5], Lc[4]);
  Lc[5] = fma(M[0], D[6], Lc[5]);
  Lc[6] = fma(M[0], D[7], Lc[6]);
  Lc[7] = fma(M[0], D[8], Lc[7]);
  Lc[8] = fma(M[0], D[9], Lc[8]);
}
template <typename T>
__device__ __forceinline__ void l2p_pe1(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=1} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  ax = fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax))));
  ay = fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay))));
  az = fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az))));
}

template <typename T>
__device__ __forceinline__ T m2l0_pe1(const T* __restrict__ M, const T* __restrict__ D) {
  return fma(-M[3], D[3], fma(-M[2], D[2], fma(-M[1], D[1], fma(M[0], D[0], T(0)))));
}
template <typename T>
__device__ __forceinline__ T l2pot_pe1(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  return fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0)))))))));
}

constexpr int kNL2 = 19;  // local coefficients, image-field order 2
template <typename T>
__device__ __forceinline__ void m2l_pe2(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {
  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..3)
  Lc[0] = fma(M[9] * T(0.5), D[15], fma(M[8], D[14], fma(M[7] * T(0.5), D[13], fma(M[6], D[12], fma(M[5], D[11], fma(M[4] * T(0.5), D[10], fma(-M[3], D[6], fma(-M[2], D[5], fma(-M[1], D[4], fma(M[0], D[1], Lc[0]))))))))));
  Lc[1] = fma(M[9] * T(0.5), D[18], fma(M[8], D[17], fma(M[7] * T(0.5), D[16], fma(M[6], D[14], fma(M[5], D[13], fma(M[4] * T(0.5), D[11], fma(-M[3], D[8], fma(-M[2], D[7], fma(-M[1], D[5], fma(M[0], D[2], Lc[1]))))))))));
  Lc[2] = fma(M[9] * T(0.5), D[19], fma(M[8], D[18], fma(M[7] * T(0.5), D[17], fma(M[6], D[15], fma(M[5], D[14], fma(M[4] * T(0.5), D[12], fma(-M[3], D[9], fma(-M[2], D[8], fma(-M[1], D[6], fma(M[0], D[3], Lc[2]))))))))));
  Lc[3] = fma(-M[3], D[12], fma(-M[2], D[11], fma(-M[1], D[10], fma(M[0], D[4], Lc[3]))));
  Lc[4] = fma(-M[3], D[14], fma(-M[2], D[13], fma(-M[1], D[11], fma(M[0], D[5], Lc[4]))));
  Lc[5] = fma(-M[3], D[15], fma(-M[2], D[14], fma(-M[1], D[12], fma(M[0], D[6], Lc[5]))));
  Lc[6] = fma(-M[3], D[17], fma(-M[2], D[16], fma(-M[1], D[13], fma(M[0], D[7], Lc[6]))));
  Lc[7] = fma(-M[3], D[18], fma(-M[2], D[17], fma(-M[1], D[14], fma(M[0], D[8], Lc[7]))));
  Lc[8] = fma(-M[3], D[19], fma(-M[2], D[18], fma(-M[1], D[15], fma(M[0], D[9], Lc[8]))));
  Lc[9] = fma(M[0], D[10], Lc[9]);
  Lc[10] = fma(M[0], D[11], Lc[10]);
  Lc[11] = fma(M[0], D[12], Lc[11]);
  Lc[12] = fma(M[0], D[13], Lc[12]);
  Lc[13] = fma(M[0], D[14], Lc[13]);
  Lc[14] = fma(M[0], D[15], Lc[14]);
  Lc[15] = fma(M[0], D[16], Lc[15]);
  Lc[16] = fma(M[0], D[17], Lc[16]);
  Lc[17] = fma(M[0], D[18], Lc[17]);
  Lc[18] = fma(M[0], D[19], Lc[18]);
}
template <typename T>
__device__ __forceinline__ void l2p_pe2(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=2} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  ax = fma(-q9, Lc[14], fma(-q8, Lc[13], fma(-q7, Lc[12], fma(-q6, Lc[11], fma(-q5, Lc[10], fma(-q4, Lc[9], fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax))))))))));
  ay = fma(-q9, Lc[17], fma(-q8, Lc[16], fma(-q7, Lc[15], fma(-q6, Lc[13], fma(-q5, Lc[12], fma(-q4, Lc[10], fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay))))))))));
  az = fma(-q9, Lc[18], fma(-q8, Lc[17], fma(-q7, Lc[16], fma(-q6, Lc[14], fma(-q5, Lc[13], fma(-q4, Lc[11], fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az))))))))));
}

template <typename T>
__device__ __forceinline__ T m2l0_pe2(const T* __restrict__ M, const T* __restrict__ D) {
  return fma(M[9] * T(0.5), D[9], fma(M[8], D[8], fma(M[7] * T(0.5), D[7], fma(M[6], D[6], fma(M[5], D[5], fma(M[4] * T(0.5), D[4], fma(-M[3], D[3], fma(-M[2], D[2], fma(-M[1], D[1], fma(M[0], D[0], T(0)))))))))));
}
template <typename T>
__device__ __forceinline__ T l2pot_pe2(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  return fma(q19, Lc[18], fma(q18, Lc[17], fma(q17, Lc[16], fma(q16, Lc[15], fma(q15, Lc[14], fma(q14, Lc[13], fma(q13, Lc[12], fma(q12, Lc[11], fma(q11, Lc[10], fma(q10, Lc[9], fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0)))))))))))))))))));
}

constexpr int kNL3 = 34;  // local coefficients, image-field order 3
template <typename T>
__device__ __forceinline__ void m2l_pe3(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {
  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..4)
  Lc[0] = fma(M[19] * T(-0.16666666666666666), D[29], fma(M[18] * T(-0.5), D[28], fma(M[17] * T(-0.5), D[27], fma(M[16] * T(-0.16666666666666666), D[26], fma(M[15] * T(-0.5), D[25], fma(-M[14], D[24], fma(M[13] * T(-0.5), D[23], fma(M[12] * T(-0.5), D[22], fma(M[11] * T(-0.5), D[21], fma(M[10] * T(-0.16666666666666666), D[20], fma(M[9] * T(0.5), D[15], fma(M[8], D[14], fma(M[7] * T(0.5), D[13], fma(M[6], D[12], fma(M[5], D[11], fma(M[4] * T(0.5), D[10], fma(-M[3], D[6], fma(-M[2], D[5], fma(-M[1], D[4], fma(M[0], D[1], Lc[0]))))))))))))))))))));
  Lc[1] = fma(M[19] * T(-0.16666666666666666), D[33], fma(M[18] * T(-0.5), D[32], fma(M[17] * T(-0.5), D[31], fma(M[16] * T(-0.16666666666666666), D[30], fma(M[15] * T(-0.5), D[28], fma(-M[14], D[27], fma(M[13] * T(-0.5), D[26], fma(M[12] * T(-0.5), D[24], fma(M[11] * T(-0.5), D[23], fma(M[10] * T(-0.16666666666666666), D[21], fma(M[9] * T(0.5), D[18], fma(M[8], D[17], fma(M[7] * T(0.5), D[16], fma(M[6], D[14], fma(M[5], D[13], fma(M[4] * T(0.5), D[11], fma(-M[3], D[8], fma(-M[2], D[7], fma(-M[1], D[5], fma(M[0], D[2], Lc[1]))))))))))))))))))));
  Lc[2] = fma(M[19] * T(-0.16666666666666666), D[34], fma(M[18] * T(-0.5), D[33], fma(M[17] * T(-0.5), D[32], fma(M[16] * T(-0.16666666666666666), D[31], fma(M[15] * T(-0.5), D[29], fma(-M[14], D[28], fma(M[13] * T(-0.5), D[27], fma(M[12] * T(-0.5), D[25], fma(M[11] * T(-0.5), D[24], fma(M[10] * T(-0.16666666666666666), D[22], fma(M[9] * T(0.5), D[19], fma(M[8], D[18], fma(M[7] * T(0.5), D[17], fma(M[6], D[15], fma(M[5], D[14], fma(M[4] * T(0.5), D[12], fma(-M[3], D[9], fma(-M[2], D[8], fma(-M[1], D[6], fma(M[0], D[3], Lc[2]))))))))))))))))))));
  Lc[3] = fma(M[9] * T(0.5), D[25], fma(M[8], D[24], fma(M[7] * T(0.5), D[23], fma(M[6], D[22], fma(M[5], D[21], fma(M[4] * T(0.5), D[20], fma(-M[3], D[12], fma(-M[2], D[11], fma(-M[1], D[10], fma(M[0], D[4], Lc[3]))))))))));
  Lc[4] = fma(M[9] * T(0.5), D[28], fma(M[8], D[27], fma(M[7] * T(0.5), D[26], fma(M[6], D[24], fma(M[5], D[23], fma(M[4] * T(0.5), D[21], fma(-M[3], D[14], fma(-M[2], D[13], fma(-M[1], D[11], fma(M[0], D[5], Lc[4]))))))))));
  Lc[5] = fma(M[9] * T(0.5), D[29], fma(M[8], D[28], fma(M[7] * T(0.5), D[27], fma(M[6], D[25], fma(M[5], D[24], fma(M[4] * T(0.5), D[22], fma(-M[3], D[15], fma(-M[2], D[14], fma(-M[1], D[12], fma(M[0], D[6], Lc[5]))))))))));
  Lc[6] = fma(M[9] * T(0.5), D[32], fma(M[8], D[31], fma(M[7] * T(0.5), D[30], fma(M[6], D[27], fma(M[5], D[26], fma(M[4] * T(0.5), D[23], fma(-M[3], D[17], fma(-M[2], D[16], fma(-M[1], D[13], fma(M[0], D[7], Lc[6]))))))))));
  Lc[7] = fma(M[9] * T(0.5), D[33], fma(M[8], D[32], fma(M[7] * T(0.5), D[31], fma(M[6], D[28], fma(M[5], D[27], fma(M[4] * T(0.5), D[24], fma(-M[3], D[18], fma(-M[2], D[17], fma(-M[1], D[14], fma(M[0], D[8], Lc[7]))))))))));
  Lc[8] = fma(M[9] * T(0.5), D[34], fma(M[8], D[33], fma(M[7] * T(0.5), D[32], fma(M[6], D[29], fma(M[5], D[28], fma(M[4] * T(0.5), D[25], fma(-M[3], D[19], fma(-M[2], D[18], fma(-M[1], D[15], fma(M[0], D[9], Lc[8]))))))))));
  Lc[9] = fma(-M[3], D[22], fma(-M[2], D[21], fma(-M[1], D[20], fma(M[0], D[10], Lc[9]))));
  Lc[10] = fma(-M[3], D[24], fma(-M[2], D[23], fma(-M[1], D[21], fma(M[0], D[11], Lc[10]))));
  Lc[11] = fma(-M[3], D[25], fma(-M[2], D[24], fma(-M[1], D[22], fma(M[0], D[12], Lc[11]))));
  Lc[12] = fma(-M[3], D[27], fma(-M[2], D[26], fma(-M[1], D[23], fma(M[0], D[13], Lc[12]))));
  Lc[13] = fma(-M[3], D[28], fma(-M[2], D[27], fma(-M[1], D[24], fma(M[0], D[14], Lc[13]))));
  Lc[14] = fma(-M[3], D[29], fma(-M[2], D[28], fma(-M[1], D[25], fma(M[0], D[15], Lc[14]))));
  Lc[15] = fma(-M[3], D[31], fma(-M[2], D[30], fma(-M[1], D[26], fma(M[0], D[16], Lc[15]))));
  Lc[16] = fma(-M[3], D[32], fma(-M[2], D[31], fma(-M[1], D[27], fma(M[0], D[17], Lc[16]))));
  Lc[17] = fma(-M[3], D[33], fma(-M[2], D[32], fma(-M[1], D[28], fma(M[0], D[18], Lc[17]))));
  Lc[18] = fma(-M[3], D[34], fma(-M[2], D[33], fma(-M[1], D[29], fma(M[0], D[19], Lc[18]))));
  Lc[19] = fma(M[0], D[20], Lc[19]);
  Lc[20] = fma(M[0], D[21], Lc[20]);
  Lc[21] = fma(M[0], D[22], Lc[21]);
  Lc[22] = fma(M[0], D[23], Lc[22]);
  Lc[23] = fma(M[0], D[24], Lc[23]);
  Lc[24] = fma(M[0], D[25], Lc[24]);
  Lc[25] = fma(M[0], D[26], Lc[25]);
  Lc[26] = fma(M[0], D[27], Lc[26]);
  Lc[27] = fma(M[0], D[28], Lc[27]);
  Lc[28] = fma(M[0], D[29], Lc[28]);
  Lc[29] = fma(M[0], D[30], Lc[29]);
  Lc[30] = fma(M[0], D[31], Lc[30]);
  Lc[31] = fma(M[0], D[32], Lc[31]);
  Lc[32] = fma(M[0], D[33], Lc[32]);
  Lc[33] = fma(M[0], D[34], Lc[33]);
}
template <typename T>
__device__ __forceinline__ void l2p_pe3(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=3} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  ax = fma(-q19, Lc[28], fma(-q18, Lc[27], fma(-q17, Lc[26], fma(-q16, Lc[25], fma(-q15, Lc[24], fma(-q14, Lc[23], fma(-q13, Lc[22], fma(-q12, Lc[21], fma(-q11, Lc[20], fma(-q10, Lc[19], fma(-q9, Lc[14], fma(-q8, Lc[13], fma(-q7, Lc[12], fma(-q6, Lc[11], fma(-q5, Lc[10], fma(-q4, Lc[9], fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax))))))))))))))))))));
  ay = fma(-q19, Lc[32], fma(-q18, Lc[31], fma(-q17, Lc[30], fma(-q16, Lc[29], fma(-q15, Lc[27], fma(-q14, Lc[26], fma(-q13, Lc[25], fma(-q12, Lc[23], fma(-q11, Lc[22], fma(-q10, Lc[20], fma(-q9, Lc[17], fma(-q8, Lc[16], fma(-q7, Lc[15], fma(-q6, Lc[13], fma(-q5, Lc[12], fma(-q4, Lc[10], fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay))))))))))))))))))));
  az = fma(-q19, Lc[33], fma(-q18, Lc[32], fma(-q17, Lc[31], fma(-q16, Lc[30], fma(-q15, Lc[28], fma(-q14, Lc[27], fma(-q13, Lc[26], fma(-q12, Lc[24], fma(-q11, Lc[23], fma(-q10, Lc[21], fma(-q9, Lc[18], fma(-q8, Lc[17], fma(-q7, Lc[16], fma(-q6, Lc[14], fma(-q5, Lc[13], fma(-q4, Lc[11], fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az))))))))))))))))))));
}

template <typename T>
__device__ __forceinline__ T m2l0_pe3(const T* __restrict__ M, const T* __restrict__ D) {
  return fma(M[19] * T(-0.16666666666666666), D[19], fma(M[18] * T(-0.5), D[18], fma(M[17] * T(-0.5), D[17], fma(M[16] * T(-0.16666666666666666), D[16], fma(M[15] * T(-0.5), D[15], fma(-M[14], D[14], fma(M[13] * T(-0.5), D[13], fma(M[12] * T(-0.5), D[12], fma(M[11] * T(-0.5), D[11], fma(M[10] * T(-0.16666666666666666), D[10], fma(M[9] * T(0.5), D[9], fma(M[8], D[8], fma(M[7] * T(0.5), D[7], fma(M[6], D[6], fma(M[5], D[5], fma(M[4] * T(0.5), D[4], fma(-M[3], D[3], fma(-M[2], D[2], fma(-M[1], D[1], fma(M[0], D[0], T(0)))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ T l2pot_pe3(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  return fma(q34, Lc[33], fma(q33, Lc[32], fma(q32, Lc[31], fma(q31, Lc[30], fma(q30, Lc[29], fma(q29, Lc[28], fma(q28, Lc[27], fma(q27, Lc[26], fma(q26, Lc[25], fma(q25, Lc[24], fma(q24, Lc[23], fma(q23, Lc[22], fma(q22, Lc[21], fma(q21, Lc[20], fma(q20, Lc[19], fma(q19, Lc[18], fma(q18, Lc[17], fma(q17, Lc[16], fma(q16, Lc[15], fma(q15, Lc[14], fma(q14, Lc[13], fma(q13, Lc[12], fma(q12, Lc[11], fma(q11, Lc[10], fma(q10, Lc[9], fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0))))))))))))))))))))))))))))))))));
}

constexpr int kNL4 = 55;  // local coefficients, image-field order 4
template <typename T>
__device__ __forceinline__ void m2l_pe4(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {
  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..5)
  Lc[0] = fma(M[34] * T(0.041666666666666664), D[49], fma(M[33] * T(0.16666666666666666), D[48], fma(M[32] * T(0.25), D[47], fma(M[31] * T(0.16666666666666666), D[46], fma(M[30] * T(0.041666666666666664), D[45], fma(M[29] * T(0.16666666666666666), D[44], fma(M[28] * T(0.5), D[43], fma(M[27] * T(0.5), D[42], fma(M[26] * T(0.16666666666666666), D[41], fma(M[25] * T(0.25), D[40], fma(M[24] * T(0.5), D[39], fma(M[23] * T(0.25), D[38], fma(M[22] * T(0.16666666666666666), D[37], fma(M[21] * T(0.16666666666666666), D[36], fma(M[20] * T(0.041666666666666664), D[35], fma(M[19] * T(-0.16666666666666666), D[29], fma(M[18] * T(-0.5), D[28], fma(M[17] * T(-0.5), D[27], fma(M[16] * T(-0.16666666666666666), D[26], fma(M[15] * T(-0.5), D[25], fma(-M[14], D[24], fma(M[13] * T(-0.5), D[23], fma(M[12] * T(-0.5), D[22], fma(M[11] * T(-0.5), D[21], fma(M[10] * T(-0.16666666666666666), D[20], fma(M[9] * T(0.5), D[15], fma(M[8], D[14], fma(M[7] * T(0.5), D[13], fma(M[6], D[12], fma(M[5], D[11], fma(M[4] * T(0.5), D[10], fma(-M[3], D[6], fma(-M[2], D[5], fma(-M[1], D[4], fma(M[0], D[1], Lc[0])))))))))))))))))))))))))))))))))));
  Lc[1] = fma(M[34] * T(0.041666666666666664), D[54], fma(M[33] * T(0.16666666666666666), D[53], fma(M[32] * T(0.25), D[52], fma(M[31] * T(0.16666666666666666), D[51], fma(M[30] * T(0.041666666666666664), D[50], fma(M[29] * T(0.16666666666666666), D[48], fma(M[28] * T(0.5), D[47], fma(M[27] * T(0.5), D[46], fma(M[26] * T(0.16666666666666666), D[45], fma(M[25] * T(0.25), D[43], fma(M[24] * T(0.5), D[42], fma(M[23] * T(0.25), D[41], fma(M[22] * T(0.16666666666666666), D[39], fma(M[21] * T(0.16666666666666666), D[38], fma(M[20] * T(0.041666666666666664), D[36], fma(M[19] * T(-0.16666666666666666), D[33], fma(M[18] * T(-0.5), D[32], fma(M[17] * T(-0.5), D[31], fma(M[16] * T(-0.16666666666666666), D[30], fma(M[15] * T(-0.5), D[28], fma(-M[14], D[27], fma(M[13] * T(-0.5), D[26], fma(M[12] * T(-0.5), D[24], fma(M[11] * T(-0.5), D[23], fma(M[10] * T(-0.16666666666666666), D[21], fma(M[9] * T(0.5), D[18], fma(M[8], D[17], fma(M[7] * T(0.5), D[16], fma(M[6], D[14], fma(M[5], D[13], fma(M[4] * T(0.5), D[11], fma(-M[3], D[8], fma(-M[2], D[7], fma(-M[1], D[5], fma(M[0], D[2], Lc[1])))))))))))))))))))))))))))))))))));
  Lc[2] = fma(M[34] * T(0.041666666666666664), D[55], fma(M[33] * T(0.16666666666666666), D[54], fma(M[32] * T(0.25), D[53], fma(M[31] * T(0.16666666666666666), D[52], fma(M[30] * T(0.041666666666666664), D[51], fma(M[29] * T(0.16666666666666666), D[49], fma(M[28] * T(0.5), D[48], fma(M[27] * T(0.5), D[47], fma(M[26] * T(0.16666666666666666), D[46], fma(M[25] * T(0.25), D[44], fma(M[24] * T(0.5), D[43], fma(M[23] * T(0.25), D[42], fma(M[22] * T(0.16666666666666666), D[40], fma(M[21] * T(0.16666666666666666), D[39], fma(M[20] * T(0.041666666666666664), D[37], fma(M[19] * T(-0.16666666666666666), D[34], fma(M[18] * T(-0.5), D[33], fma(M[17] * T(-0.5), D[32], fma(M[16] * T(-0.16666666666666666), D[31], fma(M[15] * T(-0.5), D[29], fma(-M[14], D[28], fma(M[13] * T(-0.5), D[27], fma(M[12] * T(-0.5), D[25], fma(M[11] * T(-0.5), D[24], fma(M[10] * T(-0.16666666666666666), D[22], fma(M[9] * T(0.5), D[19], fma(M[8], D[18], fma(M[7] * T(0.5), D[17], fma(M[6], D[15], fma(M[5], D[14], fma(M[4] * T(0.5), D[12], fma(-M[3], D[9], fma(-M[2], D[8], fma(-M[1], D[6], fma(M[0], D[3], Lc[2])))))))))))))))))))))))))))))))))));
  Lc[3] = fma(M[19] * T(-0.16666666666666666), D[44], fma(M[18] * T(-0.5), D[43], fma(M[17] * T(-0.5), D[42], fma(M[16] * T(-0.16666666666666666), D[41], fma(M[15] * T(-0.5), D[40], fma(-M[14], D[39], fma(M[13] * T(-0.5), D[38], fma(M[12] * T(-0.5), D[37], fma(M[11] * T(-0.5), D[36], fma(M[10] * T(-0.16666666666666666), D[35], fma(M[9] * T(0.5), D[25], fma(M[8], D[24], fma(M[7] * T(0.5), D[23], fma(M[6], D[22], fma(M[5], D[21], fma(M[4] * T(0.5), D[20], fma(-M[3], D[12], fma(-M[2], D[11], fma(-M[1], D[10], fma(M[0], D[4], Lc[3]))))))))))))))))))));
  Lc[4] = fma(M[19] * T(-0.16666666666666666), D[48], fma(M[18] * T(-0.5), D[47], fma(M[17] * T(-0.5), D[46], fma(M[16] * T(-0.16666666666666666), D[45], fma(M[15] * T(-0.5), D[43], fma(-M[14], D[42], fma(M[13] * T(-0.5), D[41], fma(M[12] * T(-0.5), D[39], fma(M[11] * T(-0.5), D[38], fma(M[10] * T(-0.16666666666666666), D[36], fma(M[9] * T(0.5), D[28], fma(M[8], D[27], fma(M[7] * T(0.5), D[26], fma(M[6], D[24], fma(M[5], D[23], fma(M[4] * T(0.5), D[21], fma(-M[3], D[14], fma(-M[2], D[13], fma(-M[1], D[11], fma(M[0], D[5], Lc[4]))))))))))))))))))));
  Lc[5] = fma(M[19] * T(-0.16666666666666666), D[49], fma(M[18] * T(-0.5), D[48], fma(M[17] * T(-0.5), D[47], fma(M[16] * T(-0.16666666666666666), D[46], fma(M[15] * T(-0.5), D[44], fma(-M[14], D[43], fma(M[13] * T(-0.5), D[42], fma(M[12] * T(-0.5), D[40], fma(M[11] * T(-0.5), D[39], fma(M[10] * T(-0.16666666666666666), D[37], fma(M[9] * T(0.5), D[29], fma(M[8], D[28], fma(M[7] * T(0.5), D[27], fma(M[6], D[25], fma(M[5], D[24], fma(M[4] * T(0.5), D[22], fma(-M[3], D[15], fma(-M[2], D[14], fma(-M[1], D[12], fma(M[0], D[6], Lc[5]))))))))))))))))))));
  Lc[6] = fma(M[19] * T(-0.16666666666666666), D[53], fma(M[18] * T(-0.5), D[52], fma(M[17] * T(-0.5), D[51], fma(M[16] * T(-0.16666666666666666), D[50], fma(M[15] * T(-0.5), D[47], fma(-M[14], D[46], fma(M[13] * T(-0.5), D[45], fma(M[12] * T(-0.5), D[42], fma(M[11] * T(-0.5), D[41], fma(M[10] * T(-0.16666666666666666), D[38], fma(M[9] * T(0.5), D[32], fma(M[8], D[31], fma(M[7] * T(0.5), D[30], fma(M[6], D[27], fma(M[5], D[26], fma(M[4] * T(0.5), D[23], fma(-M[3], D[17], fma(-M[2], D[16], fma(-M[1], D[13], fma(M[0], D[7], Lc[6]))))))))))))))))))));
  Lc[7] = fma(M[19] * T(-0.16666666666666666), D[54], fma(M[18] * T(-0.5), D[53], fma(M[17] * T(-0.5), D[52], fma(M[16] * T(-0.16666666666666666), D[51], fma(M[15] * T(-0.5), D[48], fma(-M[14], D[47], fma(M[13] * T(-0.5), D[46], fma(M[12] * T(-0.5), D[43], fma(M[11] * T(-0.5), D[42], fma(M[10] * T(-0.16666666666666666), D[39], fma(M[9] * T(0.5), D[33], fma(M[8], D[32], fma(M[7] * T(0.5), D[31], fma(M[6], D[28], fma(M[5], D[27], fma(M[4] * T(0.5), D[24], fma(-M[3], D[18], fma(-M[2], D[17], fma(-M[1], D[14], fma(M[0], D[8], Lc[7]))))))))))))))))))));
  Lc[8] = fma(M[19] * T(-0.16666666666666666), D[55], fma(M[18] * T(-0.5), D[54], fma(M[17] * T(-0.5), D[53], fma(M[16] * T(-0.16666666666666666), D[52], fma(M[15] * T(-0.5), D[49], fma(-M[14], D[48], fma(M[13] * T(-0.5), D[47], fma(M[12] * T(-0.5), D[44], fma(M[11] * T(-0.5), D[43], fma(M[10] * T(-0.16666666666666666), D[40], fma(M[9] * T(0.5), D[34], fma(M[8], D[33], fma(M[7] * T(0.5), D[32], fma(M[6], D[29], fma(M[5], D[28], fma(M[4] * T(0.5), D[25], fma(-M[3], D[19], fma(-M[2], D[18], fma(-M[1], D[15], fma(M[0], D[9], Lc[8]))))))))))))))))))));
  Lc[9] = fma(M[9] * T(0.5), D[40], fma(M[8], D[39], fma(M[7] * T(0.5), D[38], fma(M[6], D[37], fma(M[5], D[36], fma(M[4] * T(0.5), D[35], fma(-M[3], D[22], fma(-M[2], D[21], fma(-M[1], D[20], fma(M[0], D[10], Lc[9]))))))))));
  Lc[10] = fma(M[9] * T(0.5), D[43], fma(M[8], D[42], fma(M[7] * T(0.5), D[41], fma(M[6], D[39], fma(M[5], D[38], fma(M[4] * T(0.5), D[36], fma(-M[3], D[24], fma(-M[2], D[23], fma(-M[1], D[21], fma(M[0], D[11], Lc[10]))))))))));
  Lc[11] = fma(M[9] * T(0.5), D[44], fma(M[8], D[43], fma(M[7] * T(0.5), D[42], fma(M[6], D[40], fma(M[5], D[39], fma(M[4] * T(0.5), D[37], fma(-M[3], D[25], fma(-M[2], D[24], fma(-M[1], D[22], fma(M[0], D[12], Lc[11]))))))))));
  Lc[12] = fma(M[9] * T(0.5), D[47], fma(M[8], D[46], fma(M[7] * T(0.5), D[45], fma(M[6], D[42], fma(M[5], D[41], fma(M[4] * T(0.5), D[38], fma(-M[3], D[27], fma(-M[2], D[26], fma(-M[1], D[23], fma(M[0], D[13], Lc[12]))))))))));
  Lc[13] = fma(M[9] * T(0.5), D[48], fma(M[8], D[47], fma(M[7] * T(0.5), D[46], fma(M[6], D[43], fma(M[5], D[42], fma(M[4] * T(0.5), D[39], fma(-M[3], D[28], fma(-M[2], D[27], fma(-M[1], D[24], fma(M[0], D[14], Lc[13]))))))))));
  Lc[14] = fma(M[9] * T(0.5), D[49], fma(M[8], D[48], fma(M[7] * T(0.5), D[47], fma(M[6], D[44], fma(M[5], D[43], fma(M[4] * T(0.5), D[40], fma(-M[3], D[29], fma(-M[2], D[28], fma(-M[1], D[25], fma(M[0], D[15], Lc[14]))))))))));
  Lc[15] = fma(M[9] * T(0.5), D[52], fma(M[8], D[51], fma(M[7] * T(0.5), D[50], fma(M[6], D[46], fma(M[5], D[45], fma(M[4] * T(0.5), D[41], fma(-M[3], D[31], fma(-M[2], D[30], fma(-M[1], D[26], fma(M[0], D[16], Lc[15]))))))))));
  Lc[16] = fma(M[9] * T(0.5), D[53], fma(M[8], D[52], fma(M[7] * T(0.5), D[51], fma(M[6], D[47], fma(M[5], D[46], fma(M[4] * T(0.5), D[42], fma(-M[3], D[32], fma(-M[2], D[31], fma(-M[1], D[27], fma(M[0], D[17], Lc[16]))))))))));
  Lc[17] = fma(M[9] * T(0.5), D[54], fma(M[8], D[53], fma(M[7] * T(0.5), D[52], fma(M[6], D[48], fma(M[5], D[47], fma(M[4] * T(0.5), D[43], fma(-M[3], D[33], fma(-M[2], D[32], fma(-M[1], D[28], fma(M[0], D[18], Lc[17]))))))))));
  Lc[18] = fma(M[9] * T(0.5), D[55], fma(M[8], D[54], fma(M[7] * T(0.5), D[53], fma(M[6], D[49], fma(M[5], D[48], fma(M[4] * T(0.5), D[44], fma(-M[3], D[34], fma(-M[2], D[33], fma(-M[1], D[29], fma(M[0], D[19], Lc[18]))))))))));
  Lc[19] = fma(-M[3], D[37], fma(-M[2], D[36], fma(-M[1], D[35], fma(M[0], D[20], Lc[19]))));
  Lc[20] = fma(-M[3], D[39], fma(-M[2], D[38], fma(-M[1], D[36], fma(M[0], D[21], Lc[20]))));
  Lc[21] = fma(-M[3], D[40], fma(-M[2], D[39], fma(-M[1], D[37], fma(M[0], D[22], Lc[21]))));
  Lc[22] = fma(-M[3], D[42], fma(-M[2], D[41], fma(-M[1], D[38], fma(M[0], D[23], Lc[22]))));
  Lc[23] = fma(-M[3], D[43], fma(-M[2], D[42], fma(-M[1], D[39], fma(M[0], D[24], Lc[23]))));
  Lc[24] = fma(-M[3], D[44], fma(-M[2], D[43], fma(-M[1], D[40], fma(M[0], D[25], Lc[24]))));
  Lc[25] = fma(-M[3], D[46], fma(-M[2], D[45], fma(-M[1], D[41], fma(M[0], D[26], Lc[25]))));
  Lc[26] = fma(-M[3], D[47], fma(-M[2], D[46], fma(-M[1], D[42], fma(M[0], D[27], Lc[26]))));
  Lc[27] = fma(-M[3], D[48], fma(-M[2], D[47], fma(-M[1], D[43], fma(M[0], D[28], Lc[27]))));
  Lc[28] = fma(-M[3], D[49], fma(-M[2], D[48], fma(-M[1], D[44], fma(M[0], D[29], Lc[28]))));
  Lc[29] = fma(-M[3], D[51], fma(-M[2], D[50], fma(-M[1], D[45], fma(M[0], D[30], Lc[29]))));
  Lc[30] = fma(-M[3], D[52], fma(-M[2], D[51], fma(-M[1], D[46], fma(M[0], D[31], Lc[30]))));
  Lc[31] = fma(-M[3], D[53], fma(-M[2], D[52], fma(-M[1], D[47], fma(M[0], D[32], Lc[31]))));
  Lc[32] = fma(-M[3], D[54], fma(-M[2], D[53], fma(-M[1], D[48], fma(M[0], D[33], Lc[32]))));
  Lc[33] = fma(-M[3], D[55], fma(-M[2], D[54], fma(-M[1], D[49], fma(M[0], D[34], Lc[33]))));
  Lc[34] = fma(M[0], D[35], Lc[34]);
  Lc[35] = fma(M[0], D[36], Lc[35]);
  Lc[36] = fma(M[0], D[37], Lc[36]);
  Lc[37] = fma(M[0], D[38], Lc[37]);
  Lc[38] = fma(M[0], D[39], Lc[38]);
  Lc[39] = fma(M[0], D[40], Lc[39]);
  Lc[40] = fma(M[0], D[41], Lc[40]);
  Lc[41] = fma(M[0], D[42], Lc[41]);
  Lc[42] = fma(M[0], D[43], Lc[42]);
  Lc[43] = fma(M[0], D[44], Lc[43]);
  Lc[44] = fma(M[0], D[45], Lc[44]);
  Lc[45] = fma(M[0], D[46], Lc[45]);
  Lc[46] = fma(M[0], D[47], Lc[46]);
  Lc[47] = fma(M[0], D[48], Lc[47]);
  Lc[48] = fma(M[0], D[49], Lc[48]);
  Lc[49] = fma(M[0], D[50], Lc[49]);
  Lc[50] = fma(M[0], D[51], Lc[50]);
  Lc[51] = fma(M[0], D[52], Lc[51]);
  Lc[52] = fma(M[0], D[53], Lc[52]);
  Lc[53] = fma(M[0], D[54], Lc[53]);
  Lc[54] = fma(M[0], D[55], Lc[54]);
}
template <typename T>
__device__ __forceinline__ void l2p_pe4(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=4} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  ax = fma(-q34, Lc[48], fma(-q33, Lc[47], fma(-q32, Lc[46], fma(-q31, Lc[45], fma(-q30, Lc[44], fma(-q29, Lc[43], fma(-q28, Lc[42], fma(-q27, Lc[41], fma(-q26, Lc[40], fma(-q25, Lc[39], fma(-q24, Lc[38], fma(-q23, Lc[37], fma(-q22, Lc[36], fma(-q21, Lc[35], fma(-q20, Lc[34], fma(-q19, Lc[28], fma(-q18, Lc[27], fma(-q17, Lc[26], fma(-q16, Lc[25], fma(-q15, Lc[24], fma(-q14, Lc[23], fma(-q13, Lc[22], fma(-q12, Lc[21], fma(-q11, Lc[20], fma(-q10, Lc[19], fma(-q9, Lc[14], fma(-q8, Lc[13], fma(-q7, Lc[12], fma(-q6, Lc[11], fma(-q5, Lc[10], fma(-q4, Lc[9], fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax)))))))))))))))))))))))))))))))))));
  ay = fma(-q34, Lc[53], fma(-q33, Lc[52], fma(-q32, Lc[51], fma(-q31, Lc[50], fma(-q30, Lc[49], fma(-q29, Lc[47], fma(-q28, Lc[46], fma(-q27, Lc[45], fma(-q26, Lc[44], fma(-q25, Lc[42], fma(-q24, Lc[41], fma(-q23, Lc[40], fma(-q22, Lc[38], fma(-q21, Lc[37], fma(-q20, Lc[35], fma(-q19, Lc[32], fma(-q18, Lc[31], fma(-q17, Lc[30], fma(-q16, Lc[29], fma(-q15, Lc[27], fma(-q14, Lc[26], fma(-q13, Lc[25], fma(-q12, Lc[23], fma(-q11, Lc[22], fma(-q10, Lc[20], fma(-q9, Lc[17], fma(-q8, Lc[16], fma(-q7, Lc[15], fma(-q6, Lc[13], fma(-q5, Lc[12], fma(-q4, Lc[10], fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay)))))))))))))))))))))))))))))))))));
  az = fma(-q34, Lc[54], fma(-q33, Lc[53], fma(-q32, Lc[52], fma(-q31, Lc[51], fma(-q30, Lc[50], fma(-q29, Lc[48], fma(-q28, Lc[47], fma(-q27, Lc[46], fma(-q26, Lc[45], fma(-q25, Lc[43], fma(-q24, Lc[42], fma(-q23, Lc[41], fma(-q22, Lc[39], fma(-q21, Lc[38], fma(-q20, Lc[36], fma(-q19, Lc[33], fma(-q18, Lc[32], fma(-q17, Lc[31], fma(-q16, Lc[30], fma(-q15, Lc[28], fma(-q14, Lc[27], fma(-q13, Lc[26], fma(-q12, Lc[24], fma(-q11, Lc[23], fma(-q10, Lc[21], fma(-q9, Lc[18], fma(-q8, Lc[17], fma(-q7, Lc[16], fma(-q6, Lc[14], fma(-q5, Lc[13], fma(-q4, Lc[11], fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az)))))))))))))))))))))))))))))))))));
}

template <typename T>
__device__ __forceinline__ T m2l0_pe4(const T* __restrict__ M, const T* __restrict__ D) {
  return fma(M[34] * T(0.041666666666666664), D[34], fma(M[33] * T(0.16666666666666666), D[33], fma(M[32] * T(0.25), D[32], fma(M[31] * T(0.16666666666666666), D[31], fma(M[30] * T(0.041666666666666664), D[30], fma(M[29] * T(0.16666666666666666), D[29], fma(M[28] * T(0.5), D[28], fma(M[27] * T(0.5), D[27], fma(M[26] * T(0.16666666666666666), D[26], fma(M[25] * T(0.25), D[25], fma(M[24] * T(0.5), D[24], fma(M[23] * T(0.25), D[23], fma(M[22] * T(0.16666666666666666), D[22], fma(M[21] * T(0.16666666666666666), D[21], fma(M[20] * T(0.041666666666666664), D[20], fma(M[19] * T(-0.16666666666666666), D[19], fma(M[18] * T(-0.5), D[18], fma(M[17] * T(-0.5), D[17], fma(M[16] * T(-0.16666666666666666), D[16], fma(M[15] * T(-0.5), D[15], fma(-M[14], D[14], fma(M[13] * T(-0.5), D[13], fma(M[12] * T(-0.5), D[12], fma(M[11] * T(-0.5), D[11], fma(M[10] * T(-0.16666666666666666), D[10], fma(M[9] * T(0.5), D[9], fma(M[8], D[8], fma(M[7] * T(0.5), D[7], fma(M[6], D[6], fma(M[5], D[5], fma(M[4] * T(0.5), D[4], fma(-M[3], D[3], fma(-M[2], D[2], fma(-M[1], D[1], fma(M[0], D[0], T(0))))))))))))))))))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ T l2pot_pe4(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  const T q35 = q20 * (dx * T(0.20000000000000001));
  const T q36 = q21 * (dx * T(0.25));
  const T q37 = q22 * (dx * T(0.25));
  const T q38 = q23 * (dx * T(0.33333333333333331));
  const T q39 = q24 * (dx * T(0.33333333333333331));
  const T q40 = q25 * (dx * T(0.33333333333333331));
  const T q41 = q26 * (dx * T(0.5));
  const T q42 = q27 * (dx * T(0.5));
  const T q43 = q28 * (dx * T(0.5));
  const T q44 = q29 * (dx * T(0.5));
  const T q45 = q30 * (dx * T(1));
  const T q46 = q31 * (dx * T(1));
  const T q47 = q32 * (dx * T(1));
  const T q48 = q33 * (dx * T(1));
  const T q49 = q34 * (dx * T(1));
  const T q50 = q30 * (dy * T(0.20000000000000001));
  const T q51 = q31 * (dy * T(0.25));
  const T q52 = q32 * (dy * T(0.33333333333333331));
  const T q53 = q33 * (dy * T(0.5));
  const T q54 = q34 * (dy * T(1));
  const T q55 = q34 * (dz * T(0.20000000000000001));
  return fma(q55, Lc[54], fma(q54, Lc[53], fma(q53, Lc[52], fma(q52, Lc[51], fma(q51, Lc[50], fma(q50, Lc[49], fma(q49, Lc[48], fma(q48, Lc[47], fma(q47, Lc[46], fma(q46, Lc[45], fma(q45, Lc[44], fma(q44, Lc[43], fma(q43, Lc[42], fma(q42, Lc[41], fma(q41, Lc[40], fma(q40, Lc[39], fma(q39, Lc[38], fma(q38, Lc[37], fma(q37, Lc[36], fma(q36, Lc[35], fma(q35, Lc[34], fma(q34, Lc[33], fma(q33, Lc[32], fma(q32, Lc[31], fma(q31, Lc[30], fma(q30, Lc[29], fma(q29, Lc[28], fma(q28, Lc[27], fma(q27, Lc[26], fma(q26, Lc[25], fma(q25, Lc[24], fma(q24, Lc[23], fma(q23, Lc[22], fma(q22, Lc[21], fma(q21, Lc[20], fma(q20, Lc[19], fma(q19, Lc[18], fma(q18, Lc[17], fma(q17, Lc[16], fma(q16, Lc[15], fma(q15, Lc[14], fma(q14, Lc[13], fma(q13, Lc[12], fma(q12, Lc[11], fma(q11, Lc[10], fma(q10, Lc[9], fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0)))))))))))))))))))))))))))))))))))))))))))))))))))))));
}

constexpr int kNL5 = 83;  // local coefficients, image-field order 5
template <typename T>
__device__ __forceinline__ void m2l_pe5(const T* __restrict__ M, const T* __restrict__ D, T* __restrict__ Lc) {
  // Lc[t-1] accumulates L_m for multi-index t >= 1 (orders 1..6)
  Lc[0] = fma(M[55] * T(-0.0083333333333333332), D[76], fma(M[54] * T(-0.041666666666666664), D[75], fma(M[53] * T(-0.083333333333333329), D[74], fma(M[52] * T(-0.083333333333333329), D[73], fma(M[51] * T(-0.041666666666666664), D[72], fma(M[50] * T(-0.0083333333333333332), D[71], fma(M[49] * T(-0.041666666666666664), D[70], fma(M[48] * T(-0.16666666666666666), D[69], fma(M[47] * T(-0.25), D[68], fma(M[46] * T(-0.16666666666666666), D[67], fma(M[45] * T(-0.041666666666666664), D[66], fma(M[44] * T(-0.083333333333333329), D[65], fma(M[43] * T(-0.25), D[64], fma(M[42] * T(-0.25), D[63], fma(M[41] * T(-0.083333333333333329), D[62], fma(M[40] * T(-0.083333333333333329), D[61], fma(M[39] * T(-0.16666666666666666), D[60], fma(M[38] * T(-0.083333333333333329), D[59], fma(M[37] * T(-0.041666666666666664), D[58], fma(M[36] * T(-0.041666666666666664), D[57], fma(M[35] * T(-0.0083333333333333332), D[56], fma(M[34] * T(0.041666666666666664), D[49], fma(M[33] * T(0.16666666666666666), D[48], fma(M[32] * T(0.25), D[47], fma(M[31] * T(0.16666666666666666), D[46], fma(M[30] * T(0.041666666666666664), D[45], fma(M[29] * T(0.16666666666666666), D[44], fma(M[28] * T(0.5), D[43], fma(M[27] * T(0.5), D[42], fma(M[26] * T(0.16666666666666666), D[41], fma(M[25] * T(0.25), D[40], fma(M[24] * T(0.5), D[39], fma(M[23] * T(0.25), D[38], fma(M[22] * T(0.16666666666666666), D[37], fma(M[21] * T(0.16666666666666666), D[36], fma(M[20] * T(0.041666666666666664), D[35], fma(M[19] * T(-0.16666666666666666), D[29], fma(M[18] * T(-0.5), D[28], fma(M[17] * T(-0.5), D[27], fma(M[16] * T(-0.16666666666666666), D[26], fma(M[15] * T(-0.5), D[25], fma(-M[14], D[24], fma(M[13] * T(-0.5), D[23], fma(M[12] * T(-0.5), D[22], fma(M[11] * T(-0.5), D[21], fma(M[10] * T(-0.16666666666666666), D[20], fma(M[9] * T(0.5), D[15], fma(M[8], D[14], fma(M[7] * T(0.5), D[13], fma(M[6], D[12], fma(M[5], D[11], fma(M[4] * T(0.5), D[10], fma(-M[3], D[6], fma(-M[2], D[5], fma(-M[1], D[4], fma(M[0], D[1], Lc[0]))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  Lc[1] = fma(M[55] * T(-0.0083333333333333332), D[82], fma(M[54] * T(-0.041666666666666664), D[81], fma(M[53] * T(-0.083333333333333329), D[80], fma(M[52] * T(-0.083333333333333329), D[79], fma(M[51] * T(-0.041666666666666664), D[78], fma(M[50] * T(-0.0083333333333333332), D[77], fma(M[49] * T(-0.041666666666666664), D[75], fma(M[48] * T(-0.16666666666666666), D[74], fma(M[47] * T(-0.25), D[73], fma(M[46] * T(-0.16666666666666666), D[72], fma(M[45] * T(-0.041666666666666664), D[71], fma(M[44] * T(-0.083333333333333329), D[69], fma(M[43] * T(-0.25), D[68], fma(M[42] * T(-0.25), D[67], fma(M[41] * T(-0.083333333333333329), D[66], fma(M[40] * T(-0.083333333333333329), D[64], fma(M[39] * T(-0.16666666666666666), D[63], fma(M[38] * T(-0.083333333333333329), D[62], fma(M[37] * T(-0.041666666666666664), D[60], fma(M[36] * T(-0.041666666666666664), D[59], fma(M[35] * T(-0.0083333333333333332), D[57], fma(M[34] * T(0.041666666666666664), D[54], fma(M[33] * T(0.16666666666666666), D[53], fma(M[32] * T(0.25), D[52], fma(M[31] * T(0.16666666666666666), D[51], fma(M[30] * T(0.041666666666666664), D[50], fma(M[29] * T(0.16666666666666666), D[48], fma(M[28] * T(0.5), D[47], fma(M[27] * T(0.5), D[46], fma(M[26] * T(0.16666666666666666), D[45], fma(M[25] * T(0.25), D[43], fma(M[24] * T(0.5), D[42], fma(M[23] * T(0.25), D[41], fma(M[22] * T(0.16666666666666666), D[39], fma(M[21] * T(0.16666666666666666), D[38], fma(M[20] * T(0.041666666666666664), D[36], fma(M[19] * T(-0.16666666666666666), D[33], fma(M[18] * T(-0.5), D[32], fma(M[17] * T(-0.5), D[31], fma(M[16] * T(-0.16666666666666666), D[30], fma(M[15] * T(-0.5), D[28], fma(-M[14], D[27], fma(M[13] * T(-0.5), D[26], fma(M[12] * T(-0.5), D[24], fma(M[11] * T(-0.5), D[23], fma(M[10] * T(-0.16666666666666666), D[21], fma(M[9] * T(0.5), D[18], fma(M[8], D[17], fma(M[7] * T(0.5), D[16], fma(M[6], D[14], fma(M[5], D[13], fma(M[4] * T(0.5), D[11], fma(-M[3], D[8], fma(-M[2], D[7], fma(-M[1], D[5], fma(M[0], D[2], Lc[1]))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  Lc[2] = fma(M[55] * T(-0.0083333333333333332), D[83], fma(M[54] * T(-0.041666666666666664), D[82], fma(M[53] * T(-0.083333333333333329), D[81], fma(M[52] * T(-0.083333333333333329), D[80], fma(M[51] * T(-0.041666666666666664), D[79], fma(M[50] * T(-0.0083333333333333332), D[78], fma(M[49] * T(-0.041666666666666664), D[76], fma(M[48] * T(-0.16666666666666666), D[75], fma(M[47] * T(-0.25), D[74], fma(M[46] * T(-0.16666666666666666), D[73], fma(M[45] * T(-0.041666666666666664), D[72], fma(M[44] * T(-0.083333333333333329), D[70], fma(M[43] * T(-0.25), D[69], fma(M[42] * T(-0.25), D[68], fma(M[41] * T(-0.083333333333333329), D[67], fma(M[40] * T(-0.083333333333333329), D[65], fma(M[39] * T(-0.16666666666666666), D[64], fma(M[38] * T(-0.083333333333333329), D[63], fma(M[37] * T(-0.041666666666666664), D[61], fma(M[36] * T(-0.041666666666666664), D[60], fma(M[35] * T(-0.0083333333333333332), D[58], fma(M[34] * T(0.041666666666666664), D[55], fma(M[33] * T(0.16666666666666666), D[54], fma(M[32] * T(0.25), D[53], fma(M[31] * T(0.16666666666666666), D[52], fma(M[30] * T(0.041666666666666664), D[51], fma(M[29] * T(0.16666666666666666), D[49], fma(M[28] * T(0.5), D[48], fma(M[27] * T(0.5), D[47], fma(M[26] * T(0.16666666666666666), D[46], fma(M[25] * T(0.25), D[44], fma(M[24] * T(0.5), D[43], fma(M[23] * T(0.25), D[42], fma(M[22] * T(0.16666666666666666), D[40], fma(M[21] * T(0.16666666666666666), D[39], fma(M[20] * T(0.041666666666666664), D[37], fma(M[19] * T(-0.16666666666666666), D[34], fma(M[18] * T(-0.5), D[33], fma(M[17] * T(-0.5), D[32], fma(M[16] * T(-0.16666666666666666), D[31], fma(M[15] * T(-0.5), D[29], fma(-M[14], D[28], fma(M[13] * T(-0.5), D[27], fma(M[12] * T(-0.5), D[25], fma(M[11] * T(-0.5), D[24], fma(M[10] * T(-0.16666666666666666), D[22], fma(M[9] * T(0.5), D[19], fma(M[8], D[18], fma(M[7] * T(0.5), D[17], fma(M[6], D[15], fma(M[5], D[14], fma(M[4] * T(0.5), D[12], fma(-M[3], D[9], fma(-M[2], D[8], fma(-M[1], D[6], fma(M[0], D[3], Lc[2]))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  Lc[3] = fma(M[34] * T(0.041666666666666664), D[70], fma(M[33] * T(0.16666666666666666), D[69], fma(M[32] * T(0.25), D[68], fma(M[31] * T(0.16666666666666666), D[67], fma(M[30] * T(0.041666666666666664), D[66], fma(M[29] * T(0.16666666666666666), D[65], fma(M[28] * T(0.5), D[64], fma(M[27] * T(0.5), D[63], fma(M[26] * T(0.16666666666666666), D[62], fma(M[25] * T(0.25), D[61], fma(M[24] * T(0.5), D[60], fma(M[23] * T(0.25), D[59], fma(M[22] * T(0.16666666666666666), D[58], fma(M[21] * T(0.16666666666666666), D[57], fma(M[20] * T(0.041666666666666664), D[56], fma(M[19] * T(-0.16666666666666666), D[44], fma(M[18] * T(-0.5), D[43], fma(M[17] * T(-0.5), D[42], fma(M[16] * T(-0.16666666666666666), D[41], fma(M[15] * T(-0.5), D[40], fma(-M[14], D[39], fma(M[13] * T(-0.5), D[38], fma(M[12] * T(-0.5), D[37], fma(M[11] * T(-0.5), D[36], fma(M[10] * T(-0.16666666666666666), D[35], fma(M[9] * T(0.5), D[25], fma(M[8], D[24], fma(M[7] * T(0.5), D[23], fma(M[6], D[22], fma(M[5], D[21], fma(M[4] * T(0.5), D[20], fma(-M[3], D[12], fma(-M[2], D[11], fma(-M[1], D[10], fma(M[0], D[4], Lc[3])))))))))))))))))))))))))))))))))));
  Lc[4] = fma(M[34] * T(0.041666666666666664), D[75], fma(M[33] * T(0.16666666666666666), D[74], fma(M[32] * T(0.25), D[73], fma(M[31] * T(0.16666666666666666), D[72], fma(M[30] * T(0.041666666666666664), D[71], fma(M[29] * T(0.16666666666666666), D[69], fma(M[28] * T(0.5), D[68], fma(M[27] * T(0.5), D[67], fma(M[26] * T(0.16666666666666666), D[66], fma(M[25] * T(0.25), D[64], fma(M[24] * T(0.5), D[63], fma(M[23] * T(0.25), D[62], fma(M[22] * T(0.16666666666666666), D[60], fma(M[21] * T(0.16666666666666666), D[59], fma(M[20] * T(0.041666666666666664), D[57], fma(M[19] * T(-0.16666666666666666), D[48], fma(M[18] * T(-0.5), D[47], fma(M[17] * T(-0.5), D[46], fma(M[16] * T(-0.16666666666666666), D[45], fma(M[15] * T(-0.5), D[43], fma(-M[14], D[42], fma(M[13] * T(-0.5), D[41], fma(M[12] * T(-0.5), D[39], fma(M[11] * T(-0.5), D[38], fma(M[10] * T(-0.16666666666666666), D[36], fma(M[9] * T(0.5), D[28], fma(M[8], D[27], fma(M[7] * T(0.5), D[26], fma(M[6], D[24], fma(M[5], D[23], fma(M[4] * T(0.5), D[21], fma(-M[3], D[14], fma(-M[2], D[13], fma(-M[1], D[11], fma(M[0], D[5], Lc[4])))))))))))))))))))))))))))))))))));
  Lc[5] = fma(M[34] * T(0.041666666666666664), D[76], fma(M[33] * T(0.16666666666666666), D[75], fma(M[32] * T(0.25), D[74], fma(M[31] * T(0.16666666666666666), D[73], fma(M[30] * T(0.041666666666666664), D[72], fma(M[29] * T(0.16666666666666666), D[70], fma(M[28] * T(0.5), D[69], fma(M[27] * T(0.5), D[68], fma(M[26] * T(0.16666666666666666), D[67], fma(M[25] * T(0.25), D[65], fma(M[24] * T(0.5), D[64], fma(M[23] * T(0.25), D[63], fma(M[22] * T(0.16666666666666666), D[61], fma(M[21] * T(0.16666666666666666), D[60], fma(M[20] * T(0.041666666666666664), D[58], fma(M[19] * T(-0.16666666666666666), D[49], fma(M[18] * T(-0.5), D[48], fma(M[17] * T(-0.5), D[47], fma(M[16] * T(-0.16666666666666666), D[46], fma(M[15] * T(-0.5), D[44], fma(-M[14], D[43], fma(M[13] * T(-0.5), D[42], fma(M[12] * T(-0.5), D[40], fma(M[11] * T(-0.5), D[39], fma(M[10] * T(-0.16666666666666666), D[37], fma(M[9] * T(0.5), D[29], fma(M[8], D[28], fma(M[7] * T(0.5), D[27], fma(M[6], D[25], fma(M[5], D[24], fma(M[4] * T(0.5), D[22], fma(-M[3], D[15], fma(-M[2], D[14], fma(-M[1], D[12], fma(M[0], D[6], Lc[5])))))))))))))))))))))))))))))))))));
  Lc[6] = fma(M[34] * T(0.041666666666666664), D[81], fma(M[33] * T(0.16666666666666666), D[80], fma(M[32] * T(0.25), D[79], fma(M[31] * T(0.16666666666666666), D[78], fma(M[30] * T(0.041666666666666664), D[77], fma(M[29] * T(0.16666666666666666), D[74], fma(M[28] * T(0.5), D[73], fma(M[27] * T(0.5), D[72], fma(M[26] * T(0.16666666666666666), D[71], fma(M[25] * T(0.25), D[68], fma(M[24] * T(0.5), D[67], fma(M[23] * T(0.25), D[66], fma(M[22] * T(0.16666666666666666), D[63], fma(M[21] * T(0.16666666666666666), D[62], fma(M[20] * T(0.041666666666666664), D[59], fma(M[19] * T(-0.16666666666666666), D[53], fma(M[18] * T(-0.5), D[52], fma(M[17] * T(-0.5), D[51], fma(M[16] * T(-0.16666666666666666), D[50], fma(M[15] * T(-0.5), D[47], fma(-M[14], D[46], fma(M[13] * T(-0.5), D[45], fma(M[12] * T(-0.5), D[42], fma(M[11] * T(-0.5), D[41], fma(M[10] * T(-0.16666666666666666), D[38], fma(M[9] * T(0.5), D[32], fma(M[8], D[31], fma(M[7] * T(0.5), D[30], fma(M[6], D[27], fma(M[5], D[26], fma(M[4] * T(0.5), D[23], fma(-M[3], D[17], fma(-M[2], D[16], fma(-M[1], D[13], fma(M[0], D[7], Lc[6])))))))))))))))))))))))))))))))))));
  Lc[7] = fma(M[34] * T(0.041666666666666664), D[82], fma(M[33] * T(0.16666666666666666), D[81], fma(M[32] * T(0.25), D[80], fma(M[31] * T(0.16666666666666666), D[79], fma(M[30] * T(0.041666666666666664), D[78], fma(M[29] * T(0.16666666666666666), D[75], fma(M[28] * T(0.5), D[74], fma(M[27] * T(0.5), D[73], fma(M[26] * T(0.16666666666666666), D[72], fma(M[25] * T(0.25), D[69], fma(M[24] * T(0.5), D[68], fma(M[23] * T(0.25), D[67], fma(M[22] * T(0.16666666666666666), D[64], fma(M[21] * T(0.16666666666666666), D[63], fma(M[20] * T(0.041666666666666664), D[60], fma(M[19] * T(-0.16666666666666666), D[54], fma(M[18] * T(-0.5), D[53], fma(M[17] * T(-0.5), D[52], fma(M[16] * T(-0.16666666666666666), D[51], fma(M[15] * T(-0.5), D[48], fma(-M[14], D[47], fma(M[13] * T(-0.5), D[46], fma(M[12] * T(-0.5), D[43], fma(M[11] * T(-0.5), D[42], fma(M[10] * T(-0.16666666666666666), D[39], fma(M[9] * T(0.5), D[33], fma(M[8], D[32], fma(M[7] * T(0.5), D[31], fma(M[6], D[28], fma(M[5], D[27], fma(M[4] * T(0.5), D[24], fma(-M[3], D[18], fma(-M[2], D[17], fma(-M[1], D[14], fma(M[0], D[8], Lc[7])))))))))))))))))))))))))))))))))));
  Lc[8] = fma(M[34] * T(0.041666666666666664), D[83], fma(M[33] * T(0.16666666666666666), D[82], fma(M[32] * T(0.25), D[81], fma(M[31] * T(0.16666666666666666), D[80], fma(M[30] * T(0.041666666666666664), D[79], fma(M[29] * T(0.16666666666666666), D[76], fma(M[28] * T(0.5), D[75], fma(M[27] * T(0.5), D[74], fma(M[26] * T(0.16666666666666666), D[73], fma(M[25] * T(0.25), D[70], fma(M[24] * T(0.5), D[69], fma(M[23] * T(0.25), D[68], fma(M[22] * T(0.16666666666666666), D[65], fma(M[21] * T(0.16666666666666666), D[64], fma(M[20] * T(0.041666666666666664), D[61], fma(M[19] * T(-0.16666666666666666), D[55], fma(M[18] * T(-0.5), D[54], fma(M[17] * T(-0.5), D[53], fma(M[16] * T(-0.16666666666666666), D[52], fma(M[15] * T(-0.5), D[49], fma(-M[14], D[48], fma(M[13] * T(-0.5), D[47], fma(M[12] * T(-0.5), D[44], fma(M[11] * T(-0.5), D[43], fma(M[10] * T(-0.16666666666666666), D[40], fma(M[9] * T(0.5), D[34], fma(M[8], D[33], fma(M[7] * T(0.5), D[32], fma(M[6], D[29], fma(M[5], D[28], fma(M[4] * T(0.5), D[25], fma(-M[3], D[19], fma(-M[2], D[18], fma(-M[1], D[15], fma(M[0], D[9], Lc[8])))))))))))))))))))))))))))))))))));
  Lc[9] = fma(M[19] * T(-0.16666666666666666), D[65], fma(M[18] * T(-0.5), D[64], fma(M[17] * T(-0.5), D[63], fma(M[16] * T(-0.16666666666666666), D[62], fma(M[15] * T(-0.5), D[61], fma(-M[14], D[60], fma(M[13] * T(-0.5), D[59], fma(M[12] * T(-0.5), D[58], fma(M[11] * T(-0.5), D[57], fma(M[10] * T(-0.16666666666666666), D[56], fma(M[9] * T(0.5), D[40], fma(M[8], D[39], fma(M[7] * T(0.5), D[38], fma(M[6], D[37], fma(M[5], D[36], fma(M[4] * T(0.5), D[35], fma(-M[3], D[22], fma(-M[2], D[21], fma(-M[1], D[20], fma(M[0], D[10], Lc[9]))))))))))))))))))));
  Lc[10] = fma(M[19] * T(-0.16666666666666666), D[69], fma(M[18] * T(-0.5), D[68], fma(M[17] * T(-0.5), D[67], fma(M[16] * T(-0.16666666666666666), D[66], fma(M[15] * T(-0.5), D[64], fma(-M[14], D[63], fma(M[13] * T(-0.5), D[62], fma(M[12] * T(-0.5), D[60], fma(M[11] * T(-0.5), D[59], fma(M[10] * T(-0.16666666666666666), D[57], fma(M[9] * T(0.5), D[43], fma(M[8], D[42], fma(M[7] * T(0.5), D[41], fma(M[6], D[39], fma(M[5], D[38], fma(M[4] * T(0.5), D[36], fma(-M[3], D[24], fma(-M[2], D[23], fma(-M[1], D[21], fma(M[0], D[11], Lc[10]))))))))))))))))))));
  Lc[11] = fma(M[19] * T(-0.16666666666666666), D[70], fma(M[18] * T(-0.5), D[69], fma(M[17] * T(-0.5), D[68], fma(M[16] * T(-0.16666666666666666), D[67], fma(M[15] * T(-0.5), D[65], fma(-M[14], D[64], fma(M[13] * T(-0.5), D[63], fma(M[12] * T(-0.5), D[61], fma(M[11] * T(-0.5), D[60], fma(M[10] * T(-0.16666666666666666), D[58], fma(M[9] * T(0.5), D[44], fma(M[8], D[43], fma(M[7] * T(0.5), D[42], fma(M[6], D[40], fma(M[5], D[39], fma(M[4] * T(0.5), D[37], fma(-M[3], D[25], fma(-M[2], D[24], fma(-M[1], D[22], fma(M[0], D[12], Lc[11]))))))))))))))))))));
  Lc[12] = fma(M[19] * T(-0.16666666666666666), D[74], fma(M[18] * T(-0.5), D[73], fma(M[17] * T(-0.5), D[72], fma(M[16] * T(-0.16666666666666666), D[71], fma(M[15] * T(-0.5), D[68], fma(-M[14], D[67], fma(M[13] * T(-0.5), D[66], fma(M[12] * T(-0.5), D[63], fma(M[11] * T(-0.5), D[62], fma(M[10] * T(-0.16666666666666666), D[59], fma(M[9] * T(0.5), D[47], fma(M[8], D[46], fma(M[7] * T(0.5), D[45], fma(M[6], D[42], fma(M[5], D[41], fma(M[4] * T(0.5), D[38], fma(-M[3], D[27], fma(-M[2], D[26], fma(-M[1], D[23], fma(M[0], D[13], Lc[12]))))))))))))))))))));
  Lc[13] = fma(M[19] * T(-0.16666666666666666), D[75], fma(M[18] * T(-0.5), D[74], fma(M[17] * T(-0.5), D[73], fma(M[16] * T(-0.16666666666666666), D[72], fma(M[15] * T(-0.5), D[69], fma(-M[14], D[68], fma(M[13] * T(-0.5), D[67], fma(M[12] * T(-0.5), D[64], fma(M[11] * T(-0.5), D[63], fma(M[10] * T(-0.16666666666666666), D[60], fma(M[9] * T(0.5), D[48], fma(M[8], D[47], fma(M[7] * T(0.5), D[46], fma(M[6], D[43], fma(M[5], D[42], fma(M[4] * T(0.5), D[39], fma(-M[3], D[28], fma(-M[2], D[27], fma(-M[1], D[24], fma(M[0], D[14], Lc[13]))))))))))))))))))));
  Lc[14] = fma(M[19] * T(-0.16666666666666666), D[76], fma(M[18] * T(-0.5), D[75], fma(M[17] * T(-0.5), D[74], fma(M[16] * T(-0.16666666666666666), D[73], fma(M[15] * T(-0.5), D[70], fma(-M[14], D[69], fma(M[13] * T(-0.5), D[68], fma(M[12] * T(-0.5), D[65], fma(M[11] * T(-0.5), D[64], fma(M[10] * T(-0.16666666666666666), D[61], fma(M[9] * T(0.5), D[49], fma(M[8], D[48], fma(M[7] * T(0.5), D[47], fma(M[6], D[44], fma(M[5], D[43], fma(M[4] * T(0.5), D[40], fma(-M[3], D[29], fma(-M[2], D[28], fma(-M[1], D[25], fma(M[0], D[15], Lc[14]))))))))))))))))))));
  Lc[15] = fma(M[19] * T(-0.16666666666666666), D[80], fma(M[18] * T(-0.5), D[79], fma(M[17] * T(-0.5), D[78], fma(M[16] * T(-0.16666666666666666), D[77], fma(M[15] * T(-0.5), D[73], fma(-M[14], D[72], fma(M[13] * T(-0.5), D[71], fma(M[12] * T(-0.5), D[67], fma(M[11] * T(-0.5), D[66], fma(M[10] * T(-0.16666666666666666), D[62], fma(M[9] * T(0.5), D[52], fma(M[8], D[51], fma(M[7] * T(0.5), D[50], fma(M[6], D[46], fma(M[5], D[45], fma(M[4] * T(0.5), D[41], fma(-M[3], D[31], fma(-M[2], D[30], fma(-M[1], D[26], fma(M[0], D[16], Lc[15]))))))))))))))))))));
  Lc[16] = fma(M[19] * T(-0.16666666666666666), D[81], fma(M[18] * T(-0.5), D[80], fma(M[17] * T(-0.5), D[79], fma(M[16] * T(-0.16666666666666666), D[78], fma(M[15] * T(-0.5), D[74], fma(-M[14], D[73], fma(M[13] * T(-0.5), D[72], fma(M[12] * T(-0.5), D[68], fma(M[11] * T(-0.5), D[67], fma(M[10] * T(-0.16666666666666666), D[63], fma(M[9] * T(0.5), D[53], fma(M[8], D[52], fma(M[7] * T(0.5), D[51], fma(M[6], D[47], fma(M[5], D[46], fma(M[4] * T(0.5), D[42], fma(-M[3], D[32], fma(-M[2], D[31], fma(-M[1], D[27], fma(M[0], D[17], Lc[16]))))))))))))))))))));
  Lc[17] = fma(M[19] * T(-0.16666666666666666), D[82], fma(M[18] * T(-0.5), D[81], fma(M[17] * T(-0.5), D[80], fma(M[16] * T(-0.16666666666666666), D[79], fma(M[15] * T(-0.5), D[75], fma(-M[14], D[74], fma(M[13] * T(-0.5), D[73], fma(M[12] * T(-0.5), D[69], fma(M[11] * T(-0.5), D[68], fma(M[10] * T(-0.16666666666666666), D[64], fma(M[9] * T(0.5), D[54], fma(M[8], D[53], fma(M[7] * T(0.5), D[52], fma(M[6], D[48], fma(M[5], D[47], fma(M[4] * T(0.5), D[43], fma(-M[3], D[33], fma(-M[2], D[32], fma(-M[1], D[28], fma(M[0], D[18], Lc[17]))))))))))))))))))));
  Lc[18] = fma(M[19] * T(-0.16666666666666666), D[83], fma(M[18] * T(-0.5), D[82], fma(M[17] * T(-0.5), D[81], fma(M[16] * T(-0.16666666666666666), D[80], fma(M[15] * T(-0.5), D[76], fma(-M[14], D[75], fma(M[13] * T(-0.5), D[74], fma(M[12] * T(-0.5), D[70], fma(M[11] * T(-0.5), D[69], fma(M[10] * T(-0.16666666666666666), D[65], fma(M[9] * T(0.5), D[55], fma(M[8], D[54], fma(M[7] * T(0.5), D[53], fma(M[6], D[49], fma(M[5], D[48], fma(M[4] * T(0.5), D[44], fma(-M[3], D[34], fma(-M[2], D[33], fma(-M[1], D[29], fma(M[0], D[19], Lc[18]))))))))))))))))))));
  Lc[19] = fma(M[9] * T(0.5), D[61], fma(M[8], D[60], fma(M[7] * T(0.5), D[59], fma(M[6], D[58], fma(M[5], D[57], fma(M[4] * T(0.5), D[56], fma(-M[3], D[37], fma(-M[2], D[36], fma(-M[1], D[35], fma(M[0], D[20], Lc[19]))))))))));
  Lc[20] = fma(M[9] * T(0.5), D[64], fma(M[8], D[63], fma(M[7] * T(0.5), D[62], fma(M[6], D[60], fma(M[5], D[59], fma(M[4] * T(0.5), D[57], fma(-M[3], D[39], fma(-M[2], D[38], fma(-M[1], D[36], fma(M[0], D[21], Lc[20]))))))))));
  Lc[21] = fma(M[9] * T(0.5), D[65], fma(M[8], D[64], fma(M[7] * T(0.5), D[63], fma(M[6], D[61], fma(M[5], D[60], fma(M[4] * T(0.5), D[58], fma(-M[3], D[40], fma(-M[2], D[39], fma(-M[1], D[37], fma(M[0], D[22], Lc[21]))))))))));
  Lc[22] = fma(M[9] * T(0.5), D[68], fma(M[8], D[67], fma(M[7] * T(0.5), D[66], fma(M[6], D[63], fma(M[5], D[62], fma(M[4] * T(0.5), D[59], fma(-M[3], D[42], fma(-M[2], D[41], fma(-M[1], D[38], fma(M[0], D[23], Lc[22]))))))))));
  Lc[23] = fma(M[9] * T(0.5), D[69], fma(M[8], D[68], fma(M[7] * T(0.5), D[67], fma(M[6], D[64], fma(M[5], D[63], fma(M[4] * T(0.5), D[60], fma(-M[3], D[43], fma(-M[2], D[42], fma(-M[1], D[39], fma(M[0], D[24], Lc[23]))))))))));
  Lc[24] = fma(M[9] * T(0.5), D[70], fma(M[8], D[69], fma(M[7] * T(0.5), D[68], fma(M[6], D[65], fma(M[5], D[64], fma(M[4] * T(0.5), D[61], fma(-M[3], D[44], fma(-M[2], D[43], fma(-M[1], D[40], fma(M[0], D[25], Lc[24]))))))))));
  Lc[25] = fma(M[9] * T(0.5), D[73], fma(M[8], D[72], fma(M[7] * T(0.5), D[71], fma(M[6], D[67], fma(M[5], D[66], fma(M[4] * T(0.5), D[62], fma(-M[3], D[46], fma(-M[2], D[45], fma(-M[1], D[41], fma(M[0], D[26], Lc[25]))))))))));
  Lc[26] = fma(M[9] * T(0.5), D[74], fma(M[8], D[73], fma(M[7] * T(0.5), D[72], fma(M[6], D[68], fma(M[5], D[67], fma(M[4] * T(0.5), D[63], fma(-M[3], D[47], fma(-M[2], D[46], fma(-M[1], D[42], fma(M[0], D[27], Lc[26]))))))))));
  Lc[27] = fma(M[9] * T(0.5), D[75], fma(M[8], D[74], fma(M[7] * T(0.5), D[73], fma(M[6], D[69], fma(M[5], D[68], fma(M[4] * T(0.5), D[64], fma(-M[3], D[48], fma(-M[2], D[47], fma(-M[1], D[43], fma(M[0], D[28], Lc[27]))))))))));
  Lc[28] = fma(M[9] * T(0.5), D[76], fma(M[8], D[75], fma(M[7] * T(0.5), D[74], fma(M[6], D[70], fma(M[5], D[69], fma(M[4] * T(0.5), D[65], fma(-M[3], D[49], fma(-M[2], D[48], fma(-M[1], D[44], fma(M[0], D[29], Lc[28]))))))))));
  Lc[29] = fma(M[9] * T(0.5), D[79], fma(M[8], D[78], fma(M[7] * T(0.5), D[77], fma(M[6], D[72], fma(M[5], D[71], fma(M[4] * T(0.5), D[66], fma(-M[3], D[51], fma(-M[2], D[50], fma(-M[1], D[45], fma(M[0], D[30], Lc[29]))))))))));
  Lc[30] = fma(M[9] * T(0.5), D[80], fma(M[8], D[79], fma(M[7] * T(0.5), D[78], fma(M[6], D[73], fma(M[5], D[72], fma(M[4] * T(0.5), D[67], fma(-M[3], D[52], fma(-M[2], D[51], fma(-M[1], D[46], fma(M[0], D[31], Lc[30]))))))))));
  Lc[31] = fma(M[9] * T(0.5), D[81], fma(M[8], D[80], fma(M[7] * T(0.5), D[79], fma(M[6], D[74], fma(M[5], D[73], fma(M[4] * T(0.5), D[68], fma(-M[3], D[53], fma(-M[2], D[52], fma(-M[1], D[47], fma(M[0], D[32], Lc[31]))))))))));
  Lc[32] = fma(M[9] * T(0.5), D[82], fma(M[8], D[81], fma(M[7] * T(0.5), D[80], fma(M[6], D[75], fma(M[5], D[74], fma(M[4] * T(0.5), D[69], fma(-M[3], D[54], fma(-M[2], D[53], fma(-M[1], D[48], fma(M[0], D[33], Lc[32]))))))))));
  Lc[33] = fma(M[9] * T(0.5), D[83], fma(M[8], D[82], fma(M[7] * T(0.5), D[81], fma(M[6], D[76], fma(M[5], D[75], fma(M[4] * T(0.5), D[70], fma(-M[3], D[55], fma(-M[2], D[54], fma(-M[1], D[49], fma(M[0], D[34], Lc[33]))))))))));
  Lc[34] = fma(-M[3], D[58], fma(-M[2], D[57], fma(-M[1], D[56], fma(M[0], D[35], Lc[34]))));
  Lc[35] = fma(-M[3], D[60], fma(-M[2], D[59], fma(-M[1], D[57], fma(M[0], D[36], Lc[35]))));
  Lc[36] = fma(-M[3], D[61], fma(-M[2], D[60], fma(-M[1], D[58], fma(M[0], D[37], Lc[36]))));
  Lc[37] = fma(-M[3], D[63], fma(-M[2], D[62], fma(-M[1], D[59], fma(M[0], D[38], Lc[37]))));
  Lc[38] = fma(-M[3], D[64], fma(-M[2], D[63], fma(-M[1], D[60], fma(M[0], D[39], Lc[38]))));
  Lc[39] = fma(-M[3], D[65], fma(-M[2], D[64], fma(-M[1], D[61], fma(M[0], D[40], Lc[39]))));
  Lc[40] = fma(-M[3], D[67], fma(-M[2], D[66], fma(-M[1], D[62], fma(M[0], D[41], Lc[40]))));
  Lc[41] = fma(-M[3], D[68], fma(-M[2], D[67], fma(-M[1], D[63], fma(M[0], D[42], Lc[41]))));
  Lc[42] = fma(-M[3], D[69], fma(-M[2], D[68], fma(-M[1], D[64], fma(M[0], D[43], Lc[42]))));
  Lc[43] = fma(-M[3], D[70], fma(-M[2], D[69], fma(-M[1], D[65], fma(M[0], D[44], Lc[43]))));
  Lc[44] = fma(-M[3], D[72], fma(-M[2], D[71], fma(-M[1], D[66], fma(M[0], D[45], Lc[44]))));
  Lc[45] = fma(-M[3], D[73], fma(-M[2], D[72], fma(-M[1], D[67], fma(M[0], D[46], Lc[45]))));
  Lc[46] = fma(-M[3], D[74], fma(-M[2], D[73], fma(-M[1], D[68], fma(M[0], D[47], Lc[46]))));
  Lc[47] = fma(-M[3], D[75], fma(-M[2], D[74], fma(-M[1], D[69], fma(M[0], D[48], Lc[47]))));
  Lc[48] = fma(-M[3], D[76], fma(-M[2], D[75], fma(-M[1], D[70], fma(M[0], D[49], Lc[48]))));
  Lc[49] = fma(-M[3], D[78], fma(-M[2], D[77], fma(-M[1], D[71], fma(M[0], D[50], Lc[49]))));
  Lc[50] = fma(-M[3], D[79], fma(-M[2], D[78], fma(-M[1], D[72], fma(M[0], D[51], Lc[50]))));
  Lc[51] = fma(-M[3], D[80], fma(-M[2], D[79], fma(-M[1], D[73], fma(M[0], D[52], Lc[51]))));
  Lc[52] = fma(-M[3], D[81], fma(-M[2], D[80], fma(-M[1], D[74], fma(M[0], D[53], Lc[52]))));
  Lc[53] = fma(-M[3], D[82], fma(-M[2], D[81], fma(-M[1], D[75], fma(M[0], D[54], Lc[53]))));
  Lc[54] = fma(-M[3], D[83], fma(-M[2], D[82], fma(-M[1], D[76], fma(M[0], D[55], Lc[54]))));
  Lc[55] = fma(M[0], D[56], Lc[55]);
  Lc[56] = fma(M[0], D[57], Lc[56]);
  Lc[57] = fma(M[0], D[58], Lc[57]);
  Lc[58] = fma(M[0], D[59], Lc[58]);
  Lc[59] = fma(M[0], D[60], Lc[59]);
  Lc[60] = fma(M[0], D[61], Lc[60]);
  Lc[61] = fma(M[0], D[62], Lc[61]);
  Lc[62] = fma(M[0], D[63], Lc[62]);
  Lc[63] = fma(M[0], D[64], Lc[63]);
  Lc[64] = fma(M[0], D[65], Lc[64]);
  Lc[65] = fma(M[0], D[66], Lc[65]);
  Lc[66] = fma(M[0], D[67], Lc[66]);
  Lc[67] = fma(M[0], D[68], Lc[67]);
  Lc[68] = fma(M[0], D[69], Lc[68]);
  Lc[69] = fma(M[0], D[70], Lc[69]);
  Lc[70] = fma(M[0], D[71], Lc[70]);
  Lc[71] = fma(M[0], D[72], Lc[71]);
  Lc[72] = fma(M[0], D[73], Lc[72]);
  Lc[73] = fma(M[0], D[74], Lc[73]);
  Lc[74] = fma(M[0], D[75], Lc[74]);
  Lc[75] = fma(M[0], D[76], Lc[75]);
  Lc[76] = fma(M[0], D[77], Lc[76]);
  Lc[77] = fma(M[0], D[78], Lc[77]);
  Lc[78] = fma(M[0], D[79], Lc[78]);
  Lc[79] = fma(M[0], D[80], Lc[79]);
  Lc[80] = fma(M[0], D[81], Lc[80]);
  Lc[81] = fma(M[0], D[82], Lc[81]);
  Lc[82] = fma(M[0], D[83], Lc[82]);
}
template <typename T>
__device__ __forceinline__ void l2p_pe5(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=5} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  const T q35 = q20 * (dx * T(0.20000000000000001));
  const T q36 = q21 * (dx * T(0.25));
  const T q37 = q22 * (dx * T(0.25));
  const T q38 = q23 * (dx * T(0.33333333333333331));
  const T q39 = q24 * (dx * T(0.33333333333333331));
  const T q40 = q25 * (dx * T(0.33333333333333331));
  const T q41 = q26 * (dx * T(0.5));
  const T q42 = q27 * (dx * T(0.5));
  const T q43 = q28 * (dx * T(0.5));
  const T q44 = q29 * (dx * T(0.5));
  const T q45 = q30 * (dx * T(1));
  const T q46 = q31 * (dx * T(1));
  const T q47 = q32 * (dx * T(1));
  const T q48 = q33 * (dx * T(1));
  const T q49 = q34 * (dx * T(1));
  const T q50 = q30 * (dy * T(0.20000000000000001));
  const T q51 = q31 * (dy * T(0.25));
  const T q52 = q32 * (dy * T(0.33333333333333331));
  const T q53 = q33 * (dy * T(0.5));
  const T q54 = q34 * (dy * T(1));
  const T q55 = q34 * (dz * T(0.20000000000000001));
  ax = fma(-q55, Lc[75], fma(-q54, Lc[74], fma(-q53, Lc[73], fma(-q52, Lc[72], fma(-q51, Lc[71], fma(-q50, Lc[70], fma(-q49, Lc[69], fma(-q48, Lc[68], fma(-q47, Lc[67], fma(-q46, Lc[66], fma(-q45, Lc[65], fma(-q44, Lc[64], fma(-q43, Lc[63], fma(-q42, Lc[62], fma(-q41, Lc[61], fma(-q40, Lc[60], fma(-q39, Lc[59], fma(-q38, Lc[58], fma(-q37, Lc[57], fma(-q36, Lc[56], fma(-q35, Lc[55], fma(-q34, Lc[48], fma(-q33, Lc[47], fma(-q32, Lc[46], fma(-q31, Lc[45], fma(-q30, Lc[44], fma(-q29, Lc[43], fma(-q28, Lc[42], fma(-q27, Lc[41], fma(-q26, Lc[40], fma(-q25, Lc[39], fma(-q24, Lc[38], fma(-q23, Lc[37], fma(-q22, Lc[36], fma(-q21, Lc[35], fma(-q20, Lc[34], fma(-q19, Lc[28], fma(-q18, Lc[27], fma(-q17, Lc[26], fma(-q16, Lc[25], fma(-q15, Lc[24], fma(-q14, Lc[23], fma(-q13, Lc[22], fma(-q12, Lc[21], fma(-q11, Lc[20], fma(-q10, Lc[19], fma(-q9, Lc[14], fma(-q8, Lc[13], fma(-q7, Lc[12], fma(-q6, Lc[11], fma(-q5, Lc[10], fma(-q4, Lc[9], fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  ay = fma(-q55, Lc[81], fma(-q54, Lc[80], fma(-q53, Lc[79], fma(-q52, Lc[78], fma(-q51, Lc[77], fma(-q50, Lc[76], fma(-q49, Lc[74], fma(-q48, Lc[73], fma(-q47, Lc[72], fma(-q46, Lc[71], fma(-q45, Lc[70], fma(-q44, Lc[68], fma(-q43, Lc[67], fma(-q42, Lc[66], fma(-q41, Lc[65], fma(-q40, Lc[63], fma(-q39, Lc[62], fma(-q38, Lc[61], fma(-q37, Lc[59], fma(-q36, Lc[58], fma(-q35, Lc[56], fma(-q34, Lc[53], fma(-q33, Lc[52], fma(-q32, Lc[51], fma(-q31, Lc[50], fma(-q30, Lc[49], fma(-q29, Lc[47], fma(-q28, Lc[46], fma(-q27, Lc[45], fma(-q26, Lc[44], fma(-q25, Lc[42], fma(-q24, Lc[41], fma(-q23, Lc[40], fma(-q22, Lc[38], fma(-q21, Lc[37], fma(-q20, Lc[35], fma(-q19, Lc[32], fma(-q18, Lc[31], fma(-q17, Lc[30], fma(-q16, Lc[29], fma(-q15, Lc[27], fma(-q14, Lc[26], fma(-q13, Lc[25], fma(-q12, Lc[23], fma(-q11, Lc[22], fma(-q10, Lc[20], fma(-q9, Lc[17], fma(-q8, Lc[16], fma(-q7, Lc[15], fma(-q6, Lc[13], fma(-q5, Lc[12], fma(-q4, Lc[10], fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  az = fma(-q55, Lc[82], fma(-q54, Lc[81], fma(-q53, Lc[80], fma(-q52, Lc[79], fma(-q51, Lc[78], fma(-q50, Lc[77], fma(-q49, Lc[75], fma(-q48, Lc[74], fma(-q47, Lc[73], fma(-q46, Lc[72], fma(-q45, Lc[71], fma(-q44, Lc[69], fma(-q43, Lc[68], fma(-q42, Lc[67], fma(-q41, Lc[66], fma(-q40, Lc[64], fma(-q39, Lc[63], fma(-q38, Lc[62], fma(-q37, Lc[60], fma(-q36, Lc[59], fma(-q35, Lc[57], fma(-q34, Lc[54], fma(-q33, Lc[53], fma(-q32, Lc[52], fma(-q31, Lc[51], fma(-q30, Lc[50], fma(-q29, Lc[48], fma(-q28, Lc[47], fma(-q27, Lc[46], fma(-q26, Lc[45], fma(-q25, Lc[43], fma(-q24, Lc[42], fma(-q23, Lc[41], fma(-q22, Lc[39], fma(-q21, Lc[38], fma(-q20, Lc[36], fma(-q19, Lc[33], fma(-q18, Lc[32], fma(-q17, Lc[31], fma(-q16, Lc[30], fma(-q15, Lc[28], fma(-q14, Lc[27], fma(-q13, Lc[26], fma(-q12, Lc[24], fma(-q11, Lc[23], fma(-q10, Lc[21], fma(-q9, Lc[18], fma(-q8, Lc[17], fma(-q7, Lc[16], fma(-q6, Lc[14], fma(-q5, Lc[13], fma(-q4, Lc[11], fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}

template <typename T>
__device__ __forceinline__ T m2l0_pe5(const T* __restrict__ M, const T* __restrict__ D) {
  return fma(M[55] * T(-0.0083333333333333332), D[55], fma(M[54] * T(-0.041666666666666664), D[54], fma(M[53] * T(-0.083333333333333329), D[53], fma(M[52] * T(-0.083333333333333329), D[52], fma(M[51] * T(-0.041666666666666664), D[51], fma(M[50] * T(-0.0083333333333333332), D[50], fma(M[49] * T(-0.041666666666666664), D[49], fma(M[48] * T(-0.16666666666666666), D[48], fma(M[47] * T(-0.25), D[47], fma(M[46] * T(-0.16666666666666666), D[46], fma(M[45] * T(-0.041666666666666664), D[45], fma(M[44] * T(-0.083333333333333329), D[44], fma(M[43] * T(-0.25), D[43], fma(M[42] * T(-0.25), D[42], fma(M[41] * T(-0.083333333333333329), D[41], fma(M[40] * T(-0.083333333333333329), D[40], fma(M[39] * T(-0.16666666666666666), D[39], fma(M[38] * T(-0.083333333333333329), D[38], fma(M[37] * T(-0.041666666666666664), D[37], fma(M[36] * T(-0.041666666666666664), D[36], fma(M[35] * T(-0.0083333333333333332), D[35], fma(M[34] * T(0.041666666666666664), D[34], fma(M[33] * T(0.16666666666666666), D[33], fma(M[32] * T(0.25), D[32], fma(M[31] * T(0.16666666666666666), D[31], fma(M[30] * T(0.041666666666666664), D[30], fma(M[29] * T(0.16666666666666666), D[29], fma(M[28] * T(0.5), D[28], fma(M[27] * T(0.5), D[27], fma(M[26] * T(0.16666666666666666), D[26], fma(M[25] * T(0.25), D[25], fma(M[24] * T(0.5), D[24], fma(M[23] * T(0.25), D[23], fma(M[22] * T(0.16666666666666666), D[22], fma(M[21] * T(0.16666666666666666), D[21], fma(M[20] * T(0.041666666666666664), D[20], fma(M[19] * T(-0.16666666666666666), D[19], fma(M[18] * T(-0.5), D[18], fma(M[17] * T(-0.5), D[17], fma(M[16] * T(-0.16666666666666666), D[16], fma(M[15] * T(-0.5), D[15], fma(-M[14], D[14], fma(M[13] * T(-0.5), D[13], fma(M[12] * T(-0.5), D[12], fma(M[11] * T(-0.5), D[11], fma(M[10] * T(-0.16666666666666666), D[10], fma(M[9] * T(0.5), D[9], fma(M[8], D[8], fma(M[7] * T(0.5), D[7], fma(M[6], D[6], fma(M[5], D[5], fma(M[4] * T(0.5), D[4], fma(-M[3], D[3], fma(-M[2], D[2], fma(-M[1], D[1], fma(M[0], D[0], T(0)))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ T l2pot_pe5(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  const T q35 = q20 * (dx * T(0.20000000000000001));
  const T q36 = q21 * (dx * T(0.25));
  const T q37 = q22 * (dx * T(0.25));
  const T q38 = q23 * (dx * T(0.33333333333333331));
  const T q39 = q24 * (dx * T(0.33333333333333331));
  const T q40 = q25 * (dx * T(0.33333333333333331));
  const T q41 = q26 * (dx * T(0.5));
  const T q42 = q27 * (dx * T(0.5));
  const T q43 = q28 * (dx * T(0.5));
  const T q44 = q29 * (dx * T(0.5));
  const T q45 = q30 * (dx * T(1));
  const T q46 = q31 * (dx * T(1));
  const T q47 = q32 * (dx * T(1));
  const T q48 = q33 * (dx * T(1));
  const T q49 = q34 * (dx * T(1));
  const T q50 = q30 * (dy * T(0.20000000000000001));
  const T q51 = q31 * (dy * T(0.25));
  const T q52 = q32 * (dy * T(0.33333333333333331));
  const T q53 = q33 * (dy * T(0.5));
  const T q54 = q34 * (dy * T(1));
  const T q55 = q34 * (dz * T(0.20000000000000001));
  const T q56 = q35 * (dx * T(0.16666666666666666));
  const T q57 = q36 * (dx * T(0.20000000000000001));
  const T q58 = q37 * (dx * T(0.20000000000000001));
  const T q59 = q38 * (dx * T(0.25));
  const T q60 = q39 * (dx * T(0.25));
  const T q61 = q40 * (dx * T(0.25));
  const T q62 = q41 * (dx * T(0.33333333333333331));
  const T q63 = q42 * (dx * T(0.33333333333333331));
  const T q64 = q43 * (dx * T(0.33333333333333331));
  const T q65 = q44 * (dx * T(0.33333333333333331));
  const T q66 = q45 * (dx * T(0.5));
  const T q67 = q46 * (dx * T(0.5));
  const T q68 = q47 * (dx * T(0.5));
  const T q69 = q48 * (dx * T(0.5));
  const T q70 = q49 * (dx * T(0.5));
  const T q71 = q50 * (dx * T(1));
  const T q72 = q51 * (dx * T(1));
  const T q73 = q52 * (dx * T(1));
  const T q74 = q53 * (dx * T(1));
  const T q75 = q54 * (dx * T(1));
  const T q76 = q55 * (dx * T(1));
  const T q77 = q50 * (dy * T(0.16666666666666666));
  const T q78 = q51 * (dy * T(0.20000000000000001));
  const T q79 = q52 * (dy * T(0.25));
  const T q80 = q53 * (dy * T(0.33333333333333331));
  const T q81 = q54 * (dy * T(0.5));
  const T q82 = q55 * (dy * T(1));
  const T q83 = q55 * (dz * T(0.16666666666666666));
  return fma(q83, Lc[82], fma(q82, Lc[81], fma(q81, Lc[80], fma(q80, Lc[79], fma(q79, Lc[78], fma(q78, Lc[77], fma(q77, Lc[76], fma(q76, Lc[75], fma(q75, Lc[74], fma(q74, Lc[73], fma(q73, Lc[72], fma(q72, Lc[71], fma(q71, Lc[70], fma(q70, Lc[69], fma(q69, Lc[68], fma(q68, Lc[67], fma(q67, Lc[66], fma(q66, Lc[65], fma(q65, Lc[64], fma(q64, Lc[63], fma(q63, Lc[62], fma(q62, Lc[61], fma(q61, Lc[60], fma(q60, Lc[59], fma(q59, Lc[58], fma(q58, Lc[57], fma(q57, Lc[56], fma(q56, Lc[55], fma(q55, Lc[54], fma(q54, Lc[53], fma(q53, Lc[52], fma(q52, Lc[51], fma(q51, Lc[50], fma(q50, Lc[49], fma(q49, Lc[48], fma(q48, Lc[47], fma(q47, Lc[46], fma(q46, Lc[45], fma(q45, Lc[44], fma(q44, Lc[43], fma(q43, Lc[42], fma(q42, Lc[41], fma(q41, Lc[40], fma(q40, Lc[39], fma(q39, Lc[38], fma(q38, Lc[37], fma(q37, Lc[36], fma(q36, Lc[35], fma(q35, Lc[34], fma(q34, Lc[33], fma(q33, Lc[32], fma(q32, Lc[31], fma(q31, Lc[30], fma(q30, Lc[29], fma(q29, Lc[28], fma(q28, Lc[27], fma(q27, Lc[26], fma(q26, Lc[25], fma(q25, Lc[24], fma(q24, Lc[23], fma(q23, Lc[22], fma(q22, Lc[21], fma(q21, Lc[20], fma(q20, Lc[19], fma(q19, Lc[18], fma(q18, Lc[17], fma(q17, Lc[16], fma(q16, Lc[15], fma(q15, Lc[14], fma(q14, Lc[13], fma(q13, Lc[12], fma(q12, Lc[11], fma(q11, Lc[10], fma(q10, Lc[9], fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0)))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}

constexpr int kNL7 = 164;  // far-lattice local coefficients (orders 1..8)
template <typename T>
__device__ __forceinline__ void l2p_pe7(const T* __restrict__ Lc, T dx, T dy, T dz, T& ax, T& ay, T& az) {
  // a_k -= sum_{|n|<=7} d^n/n! L_{n+e_k}
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  const T q35 = q20 * (dx * T(0.20000000000000001));
  const T q36 = q21 * (dx * T(0.25));
  const T q37 = q22 * (dx * T(0.25));
  const T q38 = q23 * (dx * T(0.33333333333333331));
  const T q39 = q24 * (dx * T(0.33333333333333331));
  const T q40 = q25 * (dx * T(0.33333333333333331));
  const T q41 = q26 * (dx * T(0.5));
  const T q42 = q27 * (dx * T(0.5));
  const T q43 = q28 * (dx * T(0.5));
  const T q44 = q29 * (dx * T(0.5));
  const T q45 = q30 * (dx * T(1));
  const T q46 = q31 * (dx * T(1));
  const T q47 = q32 * (dx * T(1));
  const T q48 = q33 * (dx * T(1));
  const T q49 = q34 * (dx * T(1));
  const T q50 = q30 * (dy * T(0.20000000000000001));
  const T q51 = q31 * (dy * T(0.25));
  const T q52 = q32 * (dy * T(0.33333333333333331));
  const T q53 = q33 * (dy * T(0.5));
  const T q54 = q34 * (dy * T(1));
  const T q55 = q34 * (dz * T(0.20000000000000001));
  const T q56 = q35 * (dx * T(0.16666666666666666));
  const T q57 = q36 * (dx * T(0.20000000000000001));
  const T q58 = q37 * (dx * T(0.20000000000000001));
  const T q59 = q38 * (dx * T(0.25));
  const T q60 = q39 * (dx * T(0.25));
  const T q61 = q40 * (dx * T(0.25));
  const T q62 = q41 * (dx * T(0.33333333333333331));
  const T q63 = q42 * (dx * T(0.33333333333333331));
  const T q64 = q43 * (dx * T(0.33333333333333331));
  const T q65 = q44 * (dx * T(0.33333333333333331));
  const T q66 = q45 * (dx * T(0.5));
  const T q67 = q46 * (dx * T(0.5));
  const T q68 = q47 * (dx * T(0.5));
  const T q69 = q48 * (dx * T(0.5));
  const T q70 = q49 * (dx * T(0.5));
  const T q71 = q50 * (dx * T(1));
  const T q72 = q51 * (dx * T(1));
  const T q73 = q52 * (dx * T(1));
  const T q74 = q53 * (dx * T(1));
  const T q75 = q54 * (dx * T(1));
  const T q76 = q55 * (dx * T(1));
  const T q77 = q50 * (dy * T(0.16666666666666666));
  const T q78 = q51 * (dy * T(0.20000000000000001));
  const T q79 = q52 * (dy * T(0.25));
  const T q80 = q53 * (dy * T(0.33333333333333331));
  const T q81 = q54 * (dy * T(0.5));
  const T q82 = q55 * (dy * T(1));
  const T q83 = q55 * (dz * T(0.16666666666666666));
  const T q84 = q56 * (dx * T(0.14285714285714285));
  const T q85 = q57 * (dx * T(0.16666666666666666));
  const T q86 = q58 * (dx * T(0.16666666666666666));
  const T q87 = q59 * (dx * T(0.20000000000000001));
  const T q88 = q60 * (dx * T(0.20000000000000001));
  const T q89 = q61 * (dx * T(0.20000000000000001));
  const T q90 = q62 * (dx * T(0.25));
  const T q91 = q63 * (dx * T(0.25));
  const T q92 = q64 * (dx * T(0.25));
  const T q93 = q65 * (dx * T(0.25));
  const T q94 = q66 * (dx * T(0.33333333333333331));
  const T q95 = q67 * (dx * T(0.33333333333333331));
  const T q96 = q68 * (dx * T(0.33333333333333331));
  const T q97 = q69 * (dx * T(0.33333333333333331));
  const T q98 = q70 * (dx * T(0.33333333333333331));
  const T q99 = q71 * (dx * T(0.5));
  const T q100 = q72 * (dx * T(0.5));
  const T q101 = q73 * (dx * T(0.5));
  const T q102 = q74 * (dx * T(0.5));
  const T q103 = q75 * (dx * T(0.5));
  const T q104 = q76 * (dx * T(0.5));
  const T q105 = q77 * (dx * T(1));
  const T q106 = q78 * (dx * T(1));
  const T q107 = q79 * (dx * T(1));
  const T q108 = q80 * (dx * T(1));
  const T q109 = q81 * (dx * T(1));
  const T q110 = q82 * (dx * T(1));
  const T q111 = q83 * (dx * T(1));
  const T q112 = q77 * (dy * T(0.14285714285714285));
  const T q113 = q78 * (dy * T(0.16666666666666666));
  const T q114 = q79 * (dy * T(0.20000000000000001));
  const T q115 = q80 * (dy * T(0.25));
  const T q116 = q81 * (dy * T(0.33333333333333331));
  const T q117 = q82 * (dy * T(0.5));
  const T q118 = q83 * (dy * T(1));
  const T q119 = q83 * (dz * T(0.14285714285714285));
  ax = fma(-q119, Lc[154], fma(-q118, Lc[153], fma(-q117, Lc[152], fma(-q116, Lc[151], fma(-q115, Lc[150], fma(-q114, Lc[149], fma(-q113, Lc[148], fma(-q112, Lc[147], fma(-q111, Lc[146], fma(-q110, Lc[145], fma(-q109, Lc[144], fma(-q108, Lc[143], fma(-q107, Lc[142], fma(-q106, Lc[141], fma(-q105, Lc[140], fma(-q104, Lc[139], fma(-q103, Lc[138], fma(-q102, Lc[137], fma(-q101, Lc[136], fma(-q100, Lc[135], fma(-q99, Lc[134], fma(-q98, Lc[133], fma(-q97, Lc[132], fma(-q96, Lc[131], fma(-q95, Lc[130], fma(-q94, Lc[129], fma(-q93, Lc[128], fma(-q92, Lc[127], fma(-q91, Lc[126], fma(-q90, Lc[125], fma(-q89, Lc[124], fma(-q88, Lc[123], fma(-q87, Lc[122], fma(-q86, Lc[121], fma(-q85, Lc[120], fma(-q84, Lc[119], fma(-q83, Lc[110], fma(-q82, Lc[109], fma(-q81, Lc[108], fma(-q80, Lc[107], fma(-q79, Lc[106], fma(-q78, Lc[105], fma(-q77, Lc[104], fma(-q76, Lc[103], fma(-q75, Lc[102], fma(-q74, Lc[101], fma(-q73, Lc[100], fma(-q72, Lc[99], fma(-q71, Lc[98], fma(-q70, Lc[97], fma(-q69, Lc[96], fma(-q68, Lc[95], fma(-q67, Lc[94], fma(-q66, Lc[93], fma(-q65, Lc[92], fma(-q64, Lc[91], fma(-q63, Lc[90], fma(-q62, Lc[89], fma(-q61, Lc[88], fma(-q60, Lc[87], fma(-q59, Lc[86], fma(-q58, Lc[85], fma(-q57, Lc[84], fma(-q56, Lc[83], fma(-q55, Lc[75], fma(-q54, Lc[74], fma(-q53, Lc[73], fma(-q52, Lc[72], fma(-q51, Lc[71], fma(-q50, Lc[70], fma(-q49, Lc[69], fma(-q48, Lc[68], fma(-q47, Lc[67], fma(-q46, Lc[66], fma(-q45, Lc[65], fma(-q44, Lc[64], fma(-q43, Lc[63], fma(-q42, Lc[62], fma(-q41, Lc[61], fma(-q40, Lc[60], fma(-q39, Lc[59], fma(-q38, Lc[58], fma(-q37, Lc[57], fma(-q36, Lc[56], fma(-q35, Lc[55], fma(-q34, Lc[48], fma(-q33, Lc[47], fma(-q32, Lc[46], fma(-q31, Lc[45], fma(-q30, Lc[44], fma(-q29, Lc[43], fma(-q28, Lc[42], fma(-q27, Lc[41], fma(-q26, Lc[40], fma(-q25, Lc[39], fma(-q24, Lc[38], fma(-q23, Lc[37], fma(-q22, Lc[36], fma(-q21, Lc[35], fma(-q20, Lc[34], fma(-q19, Lc[28], fma(-q18, Lc[27], fma(-q17, Lc[26], fma(-q16, Lc[25], fma(-q15, Lc[24], fma(-q14, Lc[23], fma(-q13, Lc[22], fma(-q12, Lc[21], fma(-q11, Lc[20], fma(-q10, Lc[19], fma(-q9, Lc[14], fma(-q8, Lc[13], fma(-q7, Lc[12], fma(-q6, Lc[11], fma(-q5, Lc[10], fma(-q4, Lc[9], fma(-q3, Lc[5], fma(-q2, Lc[4], fma(-q1, Lc[3], fma(-q0, Lc[0], ax))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  ay = fma(-q119, Lc[162], fma(-q118, Lc[161], fma(-q117, Lc[160], fma(-q116, Lc[159], fma(-q115, Lc[158], fma(-q114, Lc[157], fma(-q113, Lc[156], fma(-q112, Lc[155], fma(-q111, Lc[153], fma(-q110, Lc[152], fma(-q109, Lc[151], fma(-q108, Lc[150], fma(-q107, Lc[149], fma(-q106, Lc[148], fma(-q105, Lc[147], fma(-q104, Lc[145], fma(-q103, Lc[144], fma(-q102, Lc[143], fma(-q101, Lc[142], fma(-q100, Lc[141], fma(-q99, Lc[140], fma(-q98, Lc[138], fma(-q97, Lc[137], fma(-q96, Lc[136], fma(-q95, Lc[135], fma(-q94, Lc[134], fma(-q93, Lc[132], fma(-q92, Lc[131], fma(-q91, Lc[130], fma(-q90, Lc[129], fma(-q89, Lc[127], fma(-q88, Lc[126], fma(-q87, Lc[125], fma(-q86, Lc[123], fma(-q85, Lc[122], fma(-q84, Lc[120], fma(-q83, Lc[117], fma(-q82, Lc[116], fma(-q81, Lc[115], fma(-q80, Lc[114], fma(-q79, Lc[113], fma(-q78, Lc[112], fma(-q77, Lc[111], fma(-q76, Lc[109], fma(-q75, Lc[108], fma(-q74, Lc[107], fma(-q73, Lc[106], fma(-q72, Lc[105], fma(-q71, Lc[104], fma(-q70, Lc[102], fma(-q69, Lc[101], fma(-q68, Lc[100], fma(-q67, Lc[99], fma(-q66, Lc[98], fma(-q65, Lc[96], fma(-q64, Lc[95], fma(-q63, Lc[94], fma(-q62, Lc[93], fma(-q61, Lc[91], fma(-q60, Lc[90], fma(-q59, Lc[89], fma(-q58, Lc[87], fma(-q57, Lc[86], fma(-q56, Lc[84], fma(-q55, Lc[81], fma(-q54, Lc[80], fma(-q53, Lc[79], fma(-q52, Lc[78], fma(-q51, Lc[77], fma(-q50, Lc[76], fma(-q49, Lc[74], fma(-q48, Lc[73], fma(-q47, Lc[72], fma(-q46, Lc[71], fma(-q45, Lc[70], fma(-q44, Lc[68], fma(-q43, Lc[67], fma(-q42, Lc[66], fma(-q41, Lc[65], fma(-q40, Lc[63], fma(-q39, Lc[62], fma(-q38, Lc[61], fma(-q37, Lc[59], fma(-q36, Lc[58], fma(-q35, Lc[56], fma(-q34, Lc[53], fma(-q33, Lc[52], fma(-q32, Lc[51], fma(-q31, Lc[50], fma(-q30, Lc[49], fma(-q29, Lc[47], fma(-q28, Lc[46], fma(-q27, Lc[45], fma(-q26, Lc[44], fma(-q25, Lc[42], fma(-q24, Lc[41], fma(-q23, Lc[40], fma(-q22, Lc[38], fma(-q21, Lc[37], fma(-q20, Lc[35], fma(-q19, Lc[32], fma(-q18, Lc[31], fma(-q17, Lc[30], fma(-q16, Lc[29], fma(-q15, Lc[27], fma(-q14, Lc[26], fma(-q13, Lc[25], fma(-q12, Lc[23], fma(-q11, Lc[22], fma(-q10, Lc[20], fma(-q9, Lc[17], fma(-q8, Lc[16], fma(-q7, Lc[15], fma(-q6, Lc[13], fma(-q5, Lc[12], fma(-q4, Lc[10], fma(-q3, Lc[7], fma(-q2, Lc[6], fma(-q1, Lc[4], fma(-q0, Lc[1], ay))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  az = fma(-q119, Lc[163], fma(-q118, Lc[162], fma(-q117, Lc[161], fma(-q116, Lc[160], fma(-q115, Lc[159], fma(-q114, Lc[158], fma(-q113, Lc[157], fma(-q112, Lc[156], fma(-q111, Lc[154], fma(-q110, Lc[153], fma(-q109, Lc[152], fma(-q108, Lc[151], fma(-q107, Lc[150], fma(-q106, Lc[149], fma(-q105, Lc[148], fma(-q104, Lc[146], fma(-q103, Lc[145], fma(-q102, Lc[144], fma(-q101, Lc[143], fma(-q100, Lc[142], fma(-q99, Lc[141], fma(-q98, Lc[139], fma(-q97, Lc[138], fma(-q96, Lc[137], fma(-q95, Lc[136], fma(-q94, Lc[135], fma(-q93, Lc[133], fma(-q92, Lc[132], fma(-q91, Lc[131], fma(-q90, Lc[130], fma(-q89, Lc[128], fma(-q88, Lc[127], fma(-q87, Lc[126], fma(-q86, Lc[124], fma(-q85, Lc[123], fma(-q84, Lc[121], fma(-q83, Lc[118], fma(-q82, Lc[117], fma(-q81, Lc[116], fma(-q80, Lc[115], fma(-q79, Lc[114], fma(-q78, Lc[113], fma(-q77, Lc[112], fma(-q76, Lc[110], fma(-q75, Lc[109], fma(-q74, Lc[108], fma(-q73, Lc[107], fma(-q72, Lc[106], fma(-q71, Lc[105], fma(-q70, Lc[103], fma(-q69, Lc[102], fma(-q68, Lc[101], fma(-q67, Lc[100], fma(-q66, Lc[99], fma(-q65, Lc[97], fma(-q64, Lc[96], fma(-q63, Lc[95], fma(-q62, Lc[94], fma(-q61, Lc[92], fma(-q60, Lc[91], fma(-q59, Lc[90], fma(-q58, Lc[88], fma(-q57, Lc[87], fma(-q56, Lc[85], fma(-q55, Lc[82], fma(-q54, Lc[81], fma(-q53, Lc[80], fma(-q52, Lc[79], fma(-q51, Lc[78], fma(-q50, Lc[77], fma(-q49, Lc[75], fma(-q48, Lc[74], fma(-q47, Lc[73], fma(-q46, Lc[72], fma(-q45, Lc[71], fma(-q44, Lc[69], fma(-q43, Lc[68], fma(-q42, Lc[67], fma(-q41, Lc[66], fma(-q40, Lc[64], fma(-q39, Lc[63], fma(-q38, Lc[62], fma(-q37, Lc[60], fma(-q36, Lc[59], fma(-q35, Lc[57], fma(-q34, Lc[54], fma(-q33, Lc[53], fma(-q32, Lc[52], fma(-q31, Lc[51], fma(-q30, Lc[50], fma(-q29, Lc[48], fma(-q28, Lc[47], fma(-q27, Lc[46], fma(-q26, Lc[45], fma(-q25, Lc[43], fma(-q24, Lc[42], fma(-q23, Lc[41], fma(-q22, Lc[39], fma(-q21, Lc[38], fma(-q20, Lc[36], fma(-q19, Lc[33], fma(-q18, Lc[32], fma(-q17, Lc[31], fma(-q16, Lc[30], fma(-q15, Lc[28], fma(-q14, Lc[27], fma(-q13, Lc[26], fma(-q12, Lc[24], fma(-q11, Lc[23], fma(-q10, Lc[21], fma(-q9, Lc[18], fma(-q8, Lc[17], fma(-q7, Lc[16], fma(-q6, Lc[14], fma(-q5, Lc[13], fma(-q4, Lc[11], fma(-q3, Lc[8], fma(-q2, Lc[7], fma(-q1, Lc[5], fma(-q0, Lc[2], az))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}

template <typename T>
__device__ __forceinline__ T l2pot_pe7(T L0, const T* __restrict__ Lc, T dx, T dy, T dz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  const T q4 = q1 * (dx * T(0.5));
  const T q5 = q2 * (dx * T(1));
  const T q6 = q3 * (dx * T(1));
  const T q7 = q2 * (dy * T(0.5));
  const T q8 = q3 * (dy * T(1));
  const T q9 = q3 * (dz * T(0.5));
  const T q10 = q4 * (dx * T(0.33333333333333331));
  const T q11 = q5 * (dx * T(0.5));
  const T q12 = q6 * (dx * T(0.5));
  const T q13 = q7 * (dx * T(1));
  const T q14 = q8 * (dx * T(1));
  const T q15 = q9 * (dx * T(1));
  const T q16 = q7 * (dy * T(0.33333333333333331));
  const T q17 = q8 * (dy * T(0.5));
  const T q18 = q9 * (dy * T(1));
  const T q19 = q9 * (dz * T(0.33333333333333331));
  const T q20 = q10 * (dx * T(0.25));
  const T q21 = q11 * (dx * T(0.33333333333333331));
  const T q22 = q12 * (dx * T(0.33333333333333331));
  const T q23 = q13 * (dx * T(0.5));
  const T q24 = q14 * (dx * T(0.5));
  const T q25 = q15 * (dx * T(0.5));
  const T q26 = q16 * (dx * T(1));
  const T q27 = q17 * (dx * T(1));
  const T q28 = q18 * (dx * T(1));
  const T q29 = q19 * (dx * T(1));
  const T q30 = q16 * (dy * T(0.25));
  const T q31 = q17 * (dy * T(0.33333333333333331));
  const T q32 = q18 * (dy * T(0.5));
  const T q33 = q19 * (dy * T(1));
  const T q34 = q19 * (dz * T(0.25));
  const T q35 = q20 * (dx * T(0.20000000000000001));
  const T q36 = q21 * (dx * T(0.25));
  const T q37 = q22 * (dx * T(0.25));
  const T q38 = q23 * (dx * T(0.33333333333333331));
  const T q39 = q24 * (dx * T(0.33333333333333331));
  const T q40 = q25 * (dx * T(0.33333333333333331));
  const T q41 = q26 * (dx * T(0.5));
  const T q42 = q27 * (dx * T(0.5));
  const T q43 = q28 * (dx * T(0.5));
  const T q44 = q29 * (dx * T(0.5));
  const T q45 = q30 * (dx * T(1));
  const T q46 = q31 * (dx * T(1));
  const T q47 = q32 * (dx * T(1));
  const T q48 = q33 * (dx * T(1));
  const T q49 = q34 * (dx * T(1));
  const T q50 = q30 * (dy * T(0.20000000000000001));
  const T q51 = q31 * (dy * T(0.25));
  const T q52 = q32 * (dy * T(0.33333333333333331));
  const T q53 = q33 * (dy * T(0.5));
  const T q54 = q34 * (dy * T(1));
  const T q55 = q34 * (dz * T(0.20000000000000001));
  const T q56 = q35 * (dx * T(0.16666666666666666));
  const T q57 = q36 * (dx * T(0.20000000000000001));
  const T q58 = q37 * (dx * T(0.20000000000000001));
  const T q59 = q38 * (dx * T(0.25));
  const T q60 = q39 * (dx * T(0.25));
  const T q61 = q40 * (dx * T(0.25));
  const T q62 = q41 * (dx * T(0.33333333333333331));
  const T q63 = q42 * (dx * T(0.33333333333333331));
  const T q64 = q43 * (dx * T(0.33333333333333331));
  const T q65 = q44 * (dx * T(0.33333333333333331));
  const T q66 = q45 * (dx * T(0.5));
  const T q67 = q46 * (dx * T(0.5));
  const T q68 = q47 * (dx * T(0.5));
  const T q69 = q48 * (dx * T(0.5));
  const T q70 = q49 * (dx * T(0.5));
  const T q71 = q50 * (dx * T(1));
  const T q72 = q51 * (dx * T(1));
  const T q73 = q52 * (dx * T(1));
  const T q74 = q53 * (dx * T(1));
  const T q75 = q54 * (dx * T(1));
  const T q76 = q55 * (dx * T(1));
  const T q77 = q50 * (dy * T(0.16666666666666666));
  const T q78 = q51 * (dy * T(0.20000000000000001));
  const T q79 = q52 * (dy * T(0.25));
  const T q80 = q53 * (dy * T(0.33333333333333331));
  const T q81 = q54 * (dy * T(0.5));
  const T q82 = q55 * (dy * T(1));
  const T q83 = q55 * (dz * T(0.16666666666666666));
  const T q84 = q56 * (dx * T(0.14285714285714285));
  const T q85 = q57 * (dx * T(0.16666666666666666));
  const T q86 = q58 * (dx * T(0.16666666666666666));
  const T q87 = q59 * (dx * T(0.20000000000000001));
  const T q88 = q60 * (dx * T(0.20000000000000001));
  const T q89 = q61 * (dx * T(0.20000000000000001));
  const T q90 = q62 * (dx * T(0.25));
  const T q91 = q63 * (dx * T(0.25));
  const T q92 = q64 * (dx * T(0.25));
  const T q93 = q65 * (dx * T(0.25));
  const T q94 = q66 * (dx * T(0.33333333333333331));
  const T q95 = q67 * (dx * T(0.33333333333333331));
  const T q96 = q68 * (dx * T(0.33333333333333331));
  const T q97 = q69 * (dx * T(0.33333333333333331));
  const T q98 = q70 * (dx * T(0.33333333333333331));
  const T q99 = q71 * (dx * T(0.5));
  const T q100 = q72 * (dx * T(0.5));
  const T q101 = q73 * (dx * T(0.5));
  const T q102 = q74 * (dx * T(0.5));
  const T q103 = q75 * (dx * T(0.5));
  const T q104 = q76 * (dx * T(0.5));
  const T q105 = q77 * (dx * T(1));
  const T q106 = q78 * (dx * T(1));
  const T q107 = q79 * (dx * T(1));
  const T q108 = q80 * (dx * T(1));
  const T q109 = q81 * (dx * T(1));
  const T q110 = q82 * (dx * T(1));
  const T q111 = q83 * (dx * T(1));
  const T q112 = q77 * (dy * T(0.14285714285714285));
  const T q113 = q78 * (dy * T(0.16666666666666666));
  const T q114 = q79 * (dy * T(0.20000000000000001));
  const T q115 = q80 * (dy * T(0.25));
  const T q116 = q81 * (dy * T(0.33333333333333331));
  const T q117 = q82 * (dy * T(0.5));
  const T q118 = q83 * (dy * T(1));
  const T q119 = q83 * (dz * T(0.14285714285714285));
  const T q120 = q84 * (dx * T(0.125));
  const T q121 = q85 * (dx * T(0.14285714285714285));
  const T q122 = q86 * (dx * T(0.14285714285714285));
  const T q123 = q87 * (dx * T(0.16666666666666666));
  const T q124 = q88 * (dx * T(0.16666666666666666));
  const T q125 = q89 * (dx * T(0.16666666666666666));
  const T q126 = q90 * (dx * T(0.20000000000000001));
  const T q127 = q91 * (dx * T(0.20000000000000001));
  const T q128 = q92 * (dx * T(0.20000000000000001));
  const T q129 = q93 * (dx * T(0.20000000000000001));
  const T q130 = q94 * (dx * T(0.25));
  const T q131 = q95 * (dx * T(0.25));
  const T q132 = q96 * (dx * T(0.25));
  const T q133 = q97 * (dx * T(0.25));
  const T q134 = q98 * (dx * T(0.25));
  const T q135 = q99 * (dx * T(0.33333333333333331));
  const T q136 = q100 * (dx * T(0.33333333333333331));
  const T q137 = q101 * (dx * T(0.33333333333333331));
  const T q138 = q102 * (dx * T(0.33333333333333331));
  const T q139 = q103 * (dx * T(0.33333333333333331));
  const T q140 = q104 * (dx * T(0.33333333333333331));
  const T q141 = q105 * (dx * T(0.5));
  const T q142 = q106 * (dx * T(0.5));
  const T q143 = q107 * (dx * T(0.5));
  const T q144 = q108 * (dx * T(0.5));
  const T q145 = q109 * (dx * T(0.5));
  const T q146 = q110 * (dx * T(0.5));
  const T q147 = q111 * (dx * T(0.5));
  const T q148 = q112 * (dx * T(1));
  const T q149 = q113 * (dx * T(1));
  const T q150 = q114 * (dx * T(1));
  const T q151 = q115 * (dx * T(1));
  const T q152 = q116 * (dx * T(1));
  const T q153 = q117 * (dx * T(1));
  const T q154 = q118 * (dx * T(1));
  const T q155 = q119 * (dx * T(1));
  const T q156 = q112 * (dy * T(0.125));
  const T q157 = q113 * (dy * T(0.14285714285714285));
  const T q158 = q114 * (dy * T(0.16666666666666666));
  const T q159 = q115 * (dy * T(0.20000000000000001));
  const T q160 = q116 * (dy * T(0.25));
  const T q161 = q117 * (dy * T(0.33333333333333331));
  const T q162 = q118 * (dy * T(0.5));
  const T q163 = q119 * (dy * T(1));
  const T q164 = q119 * (dz * T(0.125));
  return fma(q164, Lc[163], fma(q163, Lc[162], fma(q162, Lc[161], fma(q161, Lc[160], fma(q160, Lc[159], fma(q159, Lc[158], fma(q158, Lc[157], fma(q157, Lc[156], fma(q156, Lc[155], fma(q155, Lc[154], fma(q154, Lc[153], fma(q153, Lc[152], fma(q152, Lc[151], fma(q151, Lc[150], fma(q150, Lc[149], fma(q149, Lc[148], fma(q148, Lc[147], fma(q147, Lc[146], fma(q146, Lc[145], fma(q145, Lc[144], fma(q144, Lc[143], fma(q143, Lc[142], fma(q142, Lc[141], fma(q141, Lc[140], fma(q140, Lc[139], fma(q139, Lc[138], fma(q138, Lc[137], fma(q137, Lc[136], fma(q136, Lc[135], fma(q135, Lc[134], fma(q134, Lc[133], fma(q133, Lc[132], fma(q132, Lc[131], fma(q131, Lc[130], fma(q130, Lc[129], fma(q129, Lc[128], fma(q128, Lc[127], fma(q127, Lc[126], fma(q126, Lc[125], fma(q125, Lc[124], fma(q124, Lc[123], fma(q123, Lc[122], fma(q122, Lc[121], fma(q121, Lc[120], fma(q120, Lc[119], fma(q119, Lc[118], fma(q118, Lc[117], fma(q117, Lc[116], fma(q116, Lc[115], fma(q115, Lc[114], fma(q114, Lc[113], fma(q113, Lc[112], fma(q112, Lc[111], fma(q111, Lc[110], fma(q110, Lc[109], fma(q109, Lc[108], fma(q108, Lc[107], fma(q107, Lc[106], fma(q106, Lc[105], fma(q105, Lc[104], fma(q104, Lc[103], fma(q103, Lc[102], fma(q102, Lc[101], fma(q101, Lc[100], fma(q100, Lc[99], fma(q99, Lc[98], fma(q98, Lc[97], fma(q97, Lc[96], fma(q96, Lc[95], fma(q95, Lc[94], fma(q94, Lc[93], fma(q93, Lc[92], fma(q92, Lc[91], fma(q91, Lc[90], fma(q90, Lc[89], fma(q89, Lc[88], fma(q88, Lc[87], fma(q87, Lc[86], fma(q86, Lc[85], fma(q85, Lc[84], fma(q84, Lc[83], fma(q83, Lc[82], fma(q82, Lc[81], fma(q81, Lc[80], fma(q80, Lc[79], fma(q79, Lc[78], fma(q78, Lc[77], fma(q77, Lc[76], fma(q76, Lc[75], fma(q75, Lc[74], fma(q74, Lc[73], fma(q73, Lc[72], fma(q72, Lc[71], fma(q71, Lc[70], fma(q70, Lc[69], fma(q69, Lc[68], fma(q68, Lc[67], fma(q67, Lc[66], fma(q66, Lc[65], fma(q65, Lc[64], fma(q64, Lc[63], fma(q63, Lc[62], fma(q62, Lc[61], fma(q61, Lc[60], fma(q60, Lc[59], fma(q59, Lc[58], fma(q58, Lc[57], fma(q57, Lc[56], fma(q56, Lc[55], fma(q55, Lc[54], fma(q54, Lc[53], fma(q53, Lc[52], fma(q52, Lc[51], fma(q51, Lc[50], fma(q50, Lc[49], fma(q49, Lc[48], fma(q48, Lc[47], fma(q47, Lc[46], fma(q46, Lc[45], fma(q45, Lc[44], fma(q44, Lc[43], fma(q43, Lc[42], fma(q42, Lc[41], fma(q41, Lc[40], fma(q40, Lc[39], fma(q39, Lc[38], fma(q38, Lc[37], fma(q37, Lc[36], fma(q36, Lc[35], fma(q35, Lc[34], fma(q34, Lc[33], fma(q33, Lc[32], fma(q32, Lc[31], fma(q31, Lc[30], fma(q30, Lc[29], fma(q29, Lc[28], fma(q28, Lc[27], fma(q27, Lc[26], fma(q26, Lc[25], fma(q25, Lc[24], fma(q24, Lc[23], fma(q23, Lc[22], fma(q22, Lc[21], fma(q21, Lc[20], fma(q20, Lc[19], fma(q19, Lc[18], fma(q18, Lc[17], fma(q17, Lc[16], fma(q16, Lc[15], fma(q15, Lc[14], fma(q14, Lc[13], fma(q13, Lc[12], fma(q12, Lc[11], fma(q11, Lc[10], fma(q10, Lc[9], fma(q9, Lc[8], fma(q8, Lc[7], fma(q7, Lc[6], fma(q6, Lc[5], fma(q5, Lc[4], fma(q4, Lc[3], fma(q3, Lc[2], fma(q2, Lc[1], fma(q1, Lc[0], L0))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}

template <typename T>
__device__ __forceinline__ T m2l0_p8(const T* __restrict__ M, const T* __restrict__ D) {
  T v = T(0);
  v = fma(M[0] * T(1), D[0], v);
  v = fma(M[1] * T(-1), D[1], v);
  v = fma(M[2] * T(-1), D[2], v);
  v = fma(M[3] * T(-1), D[3], v);
  v = fma(M[4] * T(0.5), D[4], v);
  v = fma(M[5] * T(1), D[5], v);
  v = fma(M[6] * T(1), D[6], v);
  v = fma(M[7] * T(0.5), D[7], v);
  v = fma(M[8] * T(1), D[8], v);
  v = fma(M[9] * T(0.5), D[9], v);
  v = fma(M[10] * T(-0.16666666666666666), D[10], v);
  v = fma(M[11] * T(-0.5), D[11], v);
  v = fma(M[12] * T(-0.5), D[12], v);
  v = fma(M[13] * T(-0.5), D[13], v);
  v = fma(M[14] * T(-1), D[14], v);
  v = fma(M[15] * T(-0.5), D[15], v);
  v = fma(M[16] * T(-0.16666666666666666), D[16], v);
  v = fma(M[17] * T(-0.5), D[17], v);
  v = fma(M[18] * T(-0.5), D[18], v);
  v = fma(M[19] * T(-0.16666666666666666), D[19], v);
  v = fma(M[20] * T(0.041666666666666664), D[20], v);
  v = fma(M[21] * T(0.16666666666666666), D[21], v);
  v = fma(M[22] * T(0.16666666666666666), D[22], v);
  v = fma(M[23] * T(0.25), D[23], v);
  v = fma(M[24] * T(0.5), D[24], v);
  v = fma(M[25] * T(0.25), D[25], v);
  v = fma(M[26] * T(0.16666666666666666), D[26], v);
  v = fma(M[27] * T(0.5), D[27], v);
  v = fma(M[28] * T(0.5), D[28], v);
  v = fma(M[29] * T(0.16666666666666666), D[29], v);
  v = fma(M[30] * T(0.041666666666666664), D[30], v);
  v = fma(M[31] * T(0.16666666666666666), D[31], v);
  v = fma(M[32] * T(0.25), D[32], v);
  v = fma(M[33] * T(0.16666666666666666), D[33], v);
  v = fma(M[34] * T(0.041666666666666664), D[34], v);
  v = fma(M[35] * T(-0.0083333333333333332), D[35], v);
  v = fma(M[36] * T(-0.041666666666666664), D[36], v);
  v = fma(M[37] * T(-0.041666666666666664), D[37], v);
  v = fma(M[38] * T(-0.083333333333333329), D[38], v);
  v = fma(M[39] * T(-0.16666666666666666), D[39], v);
  v = fma(M[40] * T(-0.083333333333333329), D[40], v);
  v = fma(M[41] * T(-0.083333333333333329), D[41], v);
  v = fma(M[42] * T(-0.25), D[42], v);
  v = fma(M[43] * T(-0.25), D[43], v);
  v = fma(M[44] * T(-0.083333333333333329), D[44], v);
  v = fma(M[45] * T(-0.041666666666666664), D[45], v);
  v = fma(M[46] * T(-0.16666666666666666), D[46], v);
  v = fma(M[47] * T(-0.25), D[47], v);
  v = fma(M[48] * T(-0.16666666666666666), D[48], v);
  v = fma(M[49] * T(-0.041666666666666664), D[49], v);
  v = fma(M[50] * T(-0.0083333333333333332), D[50], v);
  v = fma(M[51] * T(-0.041666666666666664), D[51], v);
  v = fma(M[52] * T(-0.083333333333333329), D[52], v);
  v = fma(M[53] * T(-0.083333333333333329), D[53], v);
  v = fma(M[54] * T(-0.041666666666666664), D[54], v);
  v = fma(M[55] * T(-0.0083333333333333332), D[55], v);
  v = fma(M[56] * T(0.0013888888888888889), D[56], v);
  v = fma(M[57] * T(0.0083333333333333332), D[57], v);
  v = fma(M[58] * T(0.0083333333333333332), D[58], v);
  v = fma(M[59] * T(0.020833333333333332), D[59], v);
  v = fma(M[60] * T(0.041666666666666664), D[60], v);
  v = fma(M[61] * T(0.020833333333333332), D[61], v);
  v = fma(M[62] * T(0.027777777777777776), D[62], v);
  v = fma(M[63] * T(0.083333333333333329), D[63], v);
  v = fma(M[64] * T(0.083333333333333329), D[64], v);
  v = fma(M[65] * T(0.027777777777777776), D[65], v);
  v = fma(M[66] * T(0.020833333333333332), D[66], v);
  v = fma(M[67] * T(0.083333333333333329), D[67], v);
  v = fma(M[68] * T(0.125), D[68], v);
  v = fma(M[69] * T(0.083333333333333329), D[69], v);
  v = fma(M[70] * T(0.020833333333333332), D[70], v);
  v = fma(M[71] * T(0.0083333333333333332), D[71], v);
  v = fma(M[72] * T(0.041666666666666664), D[72], v);
  v = fma(M[73] * T(0.083333333333333329), D[73], v);
  v = fma(M[74] * T(0.083333333333333329), D[74], v);
  v = fma(M[75] * T(0.041666666666666664), D[75], v);
  v = fma(M[76] * T(0.0083333333333333332), D[76], v);
  v = fma(M[77] * T(0.0013888888888888889), D[77], v);
  v = fma(M[78] * T(0.0083333333333333332), D[78], v);
  v = fma(M[79] * T(0.020833333333333332), D[79], v);
  v = fma(M[80] * T(0.027777777777777776), D[80], v);
  v = fma(M[81] * T(0.020833333333333332), D[81], v);
  v = fma(M[82] * T(0.0083333333333333332), D[82], v);
  v = fma(M[83] * T(0.0013888888888888889), D[83], v);
  v = fma(M[84] * T(-0.00019841269841269841), D[84], v);
  v = fma(M[85] * T(-0.0013888888888888889), D[85], v);
  v = fma(M[86] * T(-0.0013888888888888889), D[86], v);
  v = fma(M[87] * T(-0.0041666666666666666), D[87], v);
  v = fma(M[88] * T(-0.0083333333333333332), D[88], v);
  v = fma(M[89] * T(-0.0041666666666666666), D[89], v);
  v = fma(M[90] * T(-0.0069444444444444441), D[90], v);
  v = fma(M[91] * T(-0.020833333333333332), D[91], v);
  v = fma(M[92] * T(-0.020833333333333332), D[92], v);
  v = fma(M[93] * T(-0.0069444444444444441), D[93], v);
  v = fma(M[94] * T(-0.0069444444444444441), D[94], v);
  v = fma(M[95] * T(-0.027777777777777776), D[95], v);
  v = fma(M[96] * T(-0.041666666666666664), D[96], v);
  v = fma(M[97] * T(-0.027777777777777776), D[97], v);
  v = fma(M[98] * T(-0.0069444444444444441), D[98], v);
  v = fma(M[99] * T(-0.0041666666666666666), D[99], v);
  v = fma(M[100] * T(-0.020833333333333332), D[100], v);
  v = fma(M[101] * T(-0.041666666666666664), D[101], v);
  v = fma(M[102] * T(-0.041666666666666664), D[102], v);
  v = fma(M[103] * T(-0.020833333333333332), D[103], v);
  v = fma(M[104] * T(-0.0041666666666666666), D[104], v);
  v = fma(M[105] * T(-0.0013888888888888889), D[105], v);
  v = fma(M[106] * T(-0.0083333333333333332), D[106], v);
  v = fma(M[107] * T(-0.020833333333333332), D[107], v);
  v = fma(M[108] * T(-0.027777777777777776), D[108], v);
  v = fma(M[109] * T(-0.020833333333333332), D[109], v);
  v = fma(M[110] * T(-0.0083333333333333332), D[110], v);
  v = fma(M[111] * T(-0.0013888888888888889), D[111], v);
  v = fma(M[112] * T(-0.00019841269841269841), D[112], v);
  v = fma(M[113] * T(-0.0013888888888888889), D[113], v);
  v = fma(M[114] * T(-0.0041666666666666666), D[114], v);
  v = fma(M[115] * T(-0.0069444444444444441), D[115], v);
  v = fma(M[116] * T(-0.0069444444444444441), D[116], v);
  v = fma(M[117] * T(-0.0041666666666666666), D[117], v);
  v = fma(M[118] * T(-0.0013888888888888889), D[118], v);
  v = fma(M[119] * T(-0.00019841269841269841), D[119], v);
  v = fma(M[120] * T(2.4801587301587302e-05), D[120], v);
  v = fma(M[121] * T(0.00019841269841269841), D[121], v);
  v = fma(M[122] * T(0.00019841269841269841), D[122], v);
  v = fma(M[123] * T(0.00069444444444444447), D[123], v);
  v = fma(M[124] * T(0.0013888888888888889), D[124], v);
  v = fma(M[125] * T(0.00069444444444444447), D[125], v);
  v = fma(M[126] * T(0.0013888888888888889), D[126], v);
  v = fma(M[127] * T(0.0041666666666666666), D[127], v);
  v = fma(M[128] * T(0.0041666666666666666), D[128], v);
  v = fma(M[129] * T(0.0013888888888888889), D[129], v);
  v = fma(M[130] * T(0.001736111111111111), D[130], v);
  v = fma(M[131] * T(0.0069444444444444441), D[131], v);
  v = fma(M[132] * T(0.010416666666666666), D[132], v);
  v = fma(M[133] * T(0.0069444444444444441), D[133], v);
  v = fma(M[134] * T(0.001736111111111111), D[134], v);
  v = fma(M[135] * T(0.0013888888888888889), D[135], v);
  v = fma(M[136] * T(0.0069444444444444441), D[136], v);
  v = fma(M[137] * T(0.013888888888888888), D[137], v);
  v = fma(M[138] * T(0.013888888888888888), D[138], v);
  v = fma(M[139] * T(0.0069444444444444441), D[139], v);
  v = fma(M[140] * T(0.0013888888888888889), D[140], v);
  v = fma(M[141] * T(0.00069444444444444447), D[141], v);
  v = fma(M[142] * T(0.0041666666666666666), D[142], v);
  v = fma(M[143] * T(0.010416666666666666), D[143], v);
  v = fma(M[144] * T(0.013888888888888888), D[144], v);
  v = fma(M[145] * T(0.010416666666666666), D[145], v);
  v = fma(M[146] * T(0.0041666666666666666), D[146], v);
  v = fma(M[147] * T(0.00069444444444444447), D[147], v);
  v = fma(M[148] * T(0.00019841269841269841), D[148], v);
  v = fma(M[149] * T(0.0013888888888888889), D[149], v);
  v = fma(M[150] * T(0.0041666666666666666), D[150], v);
  v = fma(M[151] * T(0.0069444444444444441), D[151], v);
  v = fma(M[152] * T(0.0069444444444444441), D[152], v);
  v = fma(M[153] * T(0.0041666666666666666), D[153], v);
  v = fma(M[154] * T(0.0013888888888888889), D[154], v);
  v = fma(M[155] * T(0.00019841269841269841), D[155], v);
  v = fma(M[156] * T(2.4801587301587302e-05), D[156], v);
  v = fma(M[157] * T(0.00019841269841269841), D[157], v);
  v = fma(M[158] * T(0.00069444444444444447), D[158], v);
  v = fma(M[159] * T(0.0013888888888888889), D[159], v);
  v = fma(M[160] * T(0.001736111111111111), D[160], v);
  v = fma(M[161] * T(0.0013888888888888889), D[161], v);
  v = fma(M[162] * T(0.00069444444444444447), D[162], v);
  v = fma(M[163] * T(0.00019841269841269841), D[163], v);
  v = fma(M[164] * T(2.4801587301587302e-05), D[164], v);
  return v;
}

template <typename T>
__device__ __forceinline__ void dtensor_p2(T Rx, T Ry, T Rz, T eps2, T* __restrict__ D) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T g0_0 = nbody_rsqrt(s);
  const T is = g0_0 * g0_0;
  const T g1_0 = g0_0 * (T(-1) * is);
  const T g2_0 = g1_0 * (T(-3) * is);
  const T g0_1 = Rx * g1_0;
  const T g1_1 = Rx * g2_0;
  const T g0_2 = Ry * g1_0;
  const T g1_2 = Ry * g2_0;
  const T g0_3 = Rz * g1_0;
  const T g1_3 = Rz * g2_0;
  const T g0_4 = fma(T(1), g1_0, Rx * g1_1);
  const T g0_5 = Rx * g1_2;
  const T g0_6 = Rx * g1_3;
  const T g0_7 = fma(T(1), g1_0, Ry * g1_2);
  const T g0_8 = Ry * g1_3;
  const T g0_9 = fma(T(1), g1_0, Rz * g1_3);
  D[0] = g0_0;
  D[1] = g0_1;
  D[2] = g0_2;
  D[3] = g0_3;
  D[4] = g0_4;
  D[5] = g0_5;
  D[6] = g0_6;
  D[7] = g0_7;
  D[8] = g0_8;
  D[9] = g0_9;
}

template <typename T, typename MA, typename Red>
__device__ __forceinline__ void m2l_red_p1(const MA& M, const T* __restrict__ D, Red&& red) {
  red(0, 1, fma((-M[3]), D[6], fma((-M[2]), D[5], fma((-M[1]), D[4], M[0] * D[1]))));
  red(1, 1, fma((-M[3]), D[8], fma((-M[2]), D[7], fma((-M[1]), D[5], M[0] * D[2]))));
  red(2, 1, fma((-M[3]), D[9], fma((-M[2]), D[8], fma((-M[1]), D[6], M[0] * D[3]))));
  red(3, 2, M[0] * D[4]);
  red(4, 2, M[0] * D[5]);
  red(5, 2, M[0] * D[6]);
  red(6, 2, M[0] * D[7]);
  red(7, 2, M[0] * D[8]);
  red(8, 2, M[0] * D[9]);
}

template <typename T>
__device__ __forceinline__ void dtensor_p3(T Rx, T Ry, T Rz, T eps2, T* __restrict__ D) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T g0_0 = nbody_rsqrt(s);
  const T is = g0_0 * g0_0;
  const T g1_0 = g0_0 * (T(-1) * is);
  const T g2_0 = g1_0 * (T(-3) * is);
  const T g3_0 = g2_0 * (T(-5) * is);
  const T g0_1 = Rx * g1_0;
  const T g1_1 = Rx * g2_0;
  const T g2_1 = Rx * g3_0;
  const T g0_2 = Ry * g1_0;
  const T g1_2 = Ry * g2_0;
  const T g2_2 = Ry * g3_0;
  const T g0_3 = Rz * g1_0;
  const T g1_3 = Rz * g2_0;
  const T g2_3 = Rz * g3_0;
  const T g0_4 = fma(T(1), g1_0, Rx * g1_1);
  const T g1_4 = fma(T(1), g2_0, Rx * g2_1);
  const T g0_5 = Rx * g1_2;
  const T g1_5 = Rx * g2_2;
  const T g0_6 = Rx * g1_3;
  const T g1_6 = Rx * g2_3;
  const T g0_7 = fma(T(1), g1_0, Ry * g1_2);
  const T g1_7 = fma(T(1), g2_0, Ry * g2_2);
  const T g0_8 = Ry * g1_3;
  const T g1_8 = Ry * g2_3;
  const T g0_9 = fma(T(1), g1_0, Rz * g1_3);
  const T g1_9 = fma(T(1), g2_0, Rz * g2_3);
  const T g0_10 = fma(T(2), g1_1, Rx * g1_4);
  const T g0_11 = fma(T(1), g1_2, Rx * g1_5);
  const T g0_12 = fma(T(1), g1_3, Rx * g1_6);
  const T g0_13 = Rx * g1_7;
  const T g0_14 = Rx * g1_8;
  const T g0_15 = Rx * g1_9;
  const T g0_16 = fma(T(2), g1_2, Ry * g1_7);
  const T g0_17 = fma(T(1), g1_3, Ry * g1_8);
  const T g0_18 = Ry * g1_9;
  const T g0_19 = fma(T(2), g1_3, Rz * g1_9);
  D[0] = g0_0;
  D[1] = g0_1;
  D[2] = g0_2;
  D[3] = g0_3;
  D[4] = g0_4;
  D[5] = g0_5;
  D[6] = g0_6;
  D[7] = g0_7;
  D[8] = g0_8;
  D[9] = g0_9;
  D[10] = g0_10;
  D[11] = g0_11;
  D[12] = g0_12;
  D[13] = g0_13;
  D[14] = g0_14;
  D[15] = g0_15;
  D[16] = g0_16;
  D[17] = g0_17;
  D[18] = g0_18;
  D[19] = g0_19;
}

template <typename T, typename MA, typename Red>
__device__ __forceinline__ void m2l_red_p2(const MA& M, const T* __restrict__ D, Red&& red) {
  red(0, 1, fma((M[9] * T(0.5)), D[15], fma(M[8], D[14], fma((M[7] * T(0.5)), D[13], fma(M[6], D[12], fma(M[5], D[11], fma((M[4] * T(0.5)), D[10], fma((-M[3]), D[6], fma((-M[2]), D[5], fma((-M[1]), D[4], M[0] * D[1]))))))))));
  red(1, 1, fma((M[9] * T(0.5)), D[18], fma(M[8], D[17], fma((M[7] * T(0.5)), D[16], fma(M[6], D[14], fma(M[5], D[13], fma((M[4] * T(0.5)), D[11], fma((-M[3]), D[8], fma((-M[2]), D[7], fma((-M[1]), D[5], M[0] * D[2]))))))))));
  red(2, 1, fma((M[9] * T(0.5)), D[19], fma(M[8], D[18], fma((M[7] * T(0.5)), D[17], fma(M[6], D[15], fma(M[5], D[14], fma((M[4] * T(0.5)), D[12], fma((-M[3]), D[9], fma((-M[2]), D[8], fma((-M[1]), D[6], M[0] * D[3]))))))))));
  red(3, 2, fma((-M[3]), D[12], fma((-M[2]), D[11], fma((-M[1]), D[10], M[0] * D[4]))));
  red(4, 2, fma((-M[3]), D[14], fma((-M[2]), D[13], fma((-M[1]), D[11], M[0] * D[5]))));
  red(5, 2, fma((-M[3]), D[15], fma((-M[2]), D[14], fma((-M[1]), D[12], M[0] * D[6]))));
  red(6, 2, fma((-M[3]), D[17], fma((-M[2]), D[16], fma((-M[1]), D[13], M[0] * D[7]))));
  red(7, 2, fma((-M[3]), D[18], fma((-M[2]), D[17], fma((-M[1]), D[14], M[0] * D[8]))));
  red(8, 2, fma((-M[3]), D[19], fma((-M[2]), D[18], fma((-M[1]), D[15], M[0] * D[9]))));
  red(9, 3, M[0] * D[10]);
  red(10, 3, M[0] * D[11]);
  red(11, 3, M[0] * D[12]);
  red(12, 3, M[0] * D[13]);
  red(13, 3, M[0] * D[14]);
  red(14, 3, M[0] * D[15]);
  red(15, 3, M[0] * D[16]);
  red(16, 3, M[0] * D[17]);
  red(17, 3, M[0] * D[18]);
  red(18, 3, M[0] * D[19]);
}

template <typename T>
__device__ __forceinline__ void dtensor_p4(T Rx, T Ry, T Rz, T eps2, T* __restrict__ D) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T g0_0 = nbody_rsqrt(s);
  const T is = g0_0 * g0_0;
  const T g1_0 = g0_0 * (T(-1) * is);
  const T g2_0 = g1_0 * (T(-3) * is);
  const T g3_0 = g2_0 * (T(-5) * is);
  const T g4_0 = g3_0 * (T(-7) * is);
  const T g0_1 = Rx * g1_0;
  const T g1_1 = Rx * g2_0;
  const T g2_1 = Rx * g3_0;
  const T g3_1 = Rx * g4_0;
  const T g0_2 = Ry * g1_0;
  const T g1_2 = Ry * g2_0;
  const T g2_2 = Ry * g3_0;
  const T g3_2 = Ry * g4_0;
  const T g0_3 = Rz * g1_0;
  const T g1_3 = Rz * g2_0;
  const T g2_3 = Rz * g3_0;
  const T g3_3 = Rz * g4_0;
  const T g0_4 = fma(T(1), g1_0, Rx * g1_1);
  const T g1_4 = fma(T(1), g2_0, Rx * g2_1);
  const T g2_4 = fma(T(1), g3_0, Rx * g3_1);
  const T g0_5 = Rx * g1_2;
  const T g1_5 = Rx * g2_2;
  const T g2_5 = Rx * g3_2;
  const T g0_6 = Rx * g1_3;
  const T g1_6 = Rx * g2_3;
  const T g2_6 = Rx * g3_3;
  const T g0_7 = fma(T(1), g1_0, Ry * g1_2);
  const T g1_7 = fma(T(1), g2_0, Ry * g2_2);
  const T g2_7 = fma(T(1), g3_0, Ry * g3_2);
  const T g0_8 = Ry * g1_3;
  const T g1_8 = Ry * g2_3;
  const T g2_8 = Ry * g3_3;
  const T g0_9 = fma(T(1), g1_0, Rz * g1_3);
  const T g1_9 = fma(T(1), g2_0, Rz * g2_3);
  const T g2_9 = fma(T(1), g3_0, Rz * g3_3);
  const T g0_10 = fma(T(2), g1_1, Rx * g1_4);
  const T g1_10 = fma(T(2), g2_1, Rx * g2_4);
  const T g0_11 = fma(T(1), g1_2, Rx * g1_5);
  const T g1_11 = fma(T(1), g2_2, Rx * g2_5);
  const T g0_12 = fma(T(1), g1_3, Rx * g1_6);
  const T g1_12 = fma(T(1), g2_3, Rx * g2_6);
  const T g0_13 = Rx * g1_7;
  const T g1_13 = Rx * g2_7;
  const T g0_14 = Rx * g1_8;
  const T g1_14 = Rx * g2_8;
  const T g0_15 = Rx * g1_9;
  const T g1_15 = Rx * g2_9;
  const T g0_16 = fma(T(2), g1_2, Ry * g1_7);
  const T g1_16 = fma(T(2), g2_2, Ry * g2_7);
  const T g0_17 = fma(T(1), g1_3, Ry * g1_8);
  const T g1_17 = fma(T(1), g2_3, Ry * g2_8);
  const T g0_18 = Ry * g1_9;
  const T g1_18 = Ry * g2_9;
  const T g0_19 = fma(T(2), g1_3, Rz * g1_9);
  const T g1_19 = fma(T(2), g2_3, Rz * g2_9);
  const T g0_20 = fma(T(3), g1_4, Rx * g1_10);
  const T g0_21 = fma(T(2), g1_5, Rx * g1_11);
  const T g0_22 = fma(T(2), g1_6, Rx * g1_12);
  const T g0_23 = fma(T(1), g1_7, Rx * g1_13);
  const T g0_24 = fma(T(1), g1_8, Rx * g1_14);
  const T g0_25 = fma(T(1), g1_9, Rx * g1_15);
  const T g0_26 = Rx * g1_16;
  const T g0_27 = Rx * g1_17;
  const T g0_28 = Rx * g1_18;
  const T g0_29 = Rx * g1_19;
  const T g0_30 = fma(T(3), g1_7, Ry * g1_16);
  const T g0_31 = fma(T(2), g1_8, Ry * g1_17);
  const T g0_32 = fma(T(1), g1_9, Ry * g1_18);
  const T g0_33 = Ry * g1_19;
  const T g0_34 = fma(T(3), g1_9, Rz * g1_19);
  D[0] = g0_0;
  D[1] = g0_1;
  D[2] = g0_2;
  D[3] = g0_3;
  D[4] = g0_4;
  D[5] = g0_5;
  D[6] = g0_6;
  D[7] = g0_7;
  D[8] = g0_8;
  D[9] = g0_9;
  D[10] = g0_10;
  D[11] = g0_11;
  D[12] = g0_12;
  D[13] = g0_13;
  D[14] = g0_14;
  D[15] = g0_15;
  D[16] = g0_16;
  D[17] = g0_17;
  D[18] = g0_18;
  D[19] = g0_19;
  D[20] = g0_20;
  D[21] = g0_21;
  D[22] = g0_22;
  D[23] = g0_23;
  D[24] = g0_24;
  D[25] = g0_25;
  D[26] = g0_26;
  D[27] = g0_27;
  D[28] = g0_28;
  D[29] = g0_29;
  D[30] = g0_30;
  D[31] = g0_31;
  D[32] = g0_32;
  D[33] = g0_33;
  D[34] = g0_34;
}

template <typename T, typename MA, typename Red>
__device__ __forceinline__ void m2l_red_p3(const MA& M, const T* __restrict__ D, Red&& red) {
  red(0, 1, fma((M[19] * T(-0.16666666666666666)), D[29], fma((M[18] * T(-0.5)), D[28], fma((M[17] * T(-0.5)), D[27], fma((M[16] * T(-0.16666666666666666)), D[26], fma((M[15] * T(-0.5)), D[25], fma((-M[14]), D[24], fma((M[13] * T(-0.5)), D[23], fma((M[12] * T(-0.5)), D[22], fma((M[11] * T(-0.5)), D[21], fma((M[10] * T(-0.16666666666666666)), D[20], fma((M[9] * T(0.5)), D[15], fma(M[8], D[14], fma((M[7] * T(0.5)), D[13], fma(M[6], D[12], fma(M[5], D[11], fma((M[4] * T(0.5)), D[10], fma((-M[3]), D[6], fma((-M[2]), D[5], fma((-M[1]), D[4], M[0] * D[1]))))))))))))))))))));
  red(1, 1, fma((M[19] * T(-0.16666666666666666)), D[33], fma((M[18] * T(-0.5)), D[32], fma((M[17] * T(-0.5)), D[31], fma((M[16] * T(-0.16666666666666666)), D[30], fma((M[15] * T(-0.5)), D[28], fma((-M[14]), D[27], fma((M[13] * T(-0.5)), D[26], fma((M[12] * T(-0.5)), D[24], fma((M[11] * T(-0.5)), D[23], fma((M[10] * T(-0.16666666666666666)), D[21], fma((M[9] * T(0.5)), D[18], fma(M[8], D[17], fma((M[7] * T(0.5)), D[16], fma(M[6], D[14], fma(M[5], D[13], fma((M[4] * T(0.5)), D[11], fma((-M[3]), D[8], fma((-M[2]), D[7], fma((-M[1]), D[5], M[0] * D[2]))))))))))))))))))));
  red(2, 1, fma((M[19] * T(-0.16666666666666666)), D[34], fma((M[18] * T(-0.5)), D[33], fma((M[17] * T(-0.5)), D[32], fma((M[16] * T(-0.16666666666666666)), D[31], fma((M[15] * T(-0.5)), D[29], fma((-M[14]), D[28], fma((M[13] * T(-0.5)), D[27], fma((M[12] * T(-0.5)), D[25], fma((M[11] * T(-0.5)), D[24], fma((M[10] * T(-0.16666666666666666)), D[22], fma((M[9] * T(0.5)), D[19], fma(M[8], D[18], fma((M[7] * T(0.5)), D[17], fma(M[6], D[15], fma(M[5], D[14], fma((M[4] * T(0.5)), D[12], fma((-M[3]), D[9], fma((-M[2]), D[8], fma((-M[1]), D[6], M[0] * D[3]))))))))))))))))))));
  red(3, 2, fma((M[9] * T(0.5)), D[25], fma(M[8], D[24], fma((M[7] * T(0.5)), D[23], fma(M[6], D[22], fma(M[5], D[21], fma((M[4] * T(0.5)), D[20], fma((-M[3]), D[12], fma((-M[2]), D[11], fma((-M[1]), D[10], M[0] * D[4]))))))))));
  red(4, 2, fma((M[9] * T(0.5)), D[28], fma(M[8], D[27], fma((M[7] * T(0.5)), D[26], fma(M[6], D[24], fma(M[5], D[23], fma((M[4] * T(0.5)), D[21], fma((-M[3]), D[14], fma((-M[2]), D[13], fma((-M[1]), D[11], M[0] * D[5]))))))))));
  red(5, 2, fma((M[9] * T(0.5)), D[29], fma(M[8], D[28], fma((M[7] * T(0.5)), D[27], fma(M[6], D[25], fma(M[5], D[24], fma((M[4] * T(0.5)), D[22], fma((-M[3]), D[15], fma((-M[2]), D[14], fma((-M[1]), D[12], M[0] * D[6]))))))))));
  red(6, 2, fma((M[9] * T(0.5)), D[32], fma(M[8], D[31], fma((M[7] * T(0.5)), D[30], fma(M[6], D[27], fma(M[5], D[26], fma((M[4] * T(0.5)), D[23], fma((-M[3]), D[17], fma((-M[2]), D[16], fma((-M[1]), D[13], M[0] * D[7]))))))))));
  red(7, 2, fma((M[9] * T(0.5)), D[33], fma(M[8], D[32], fma((M[7] * T(0.5)), D[31], fma(M[6], D[28], fma(M[5], D[27], fma((M[4] * T(0.5)), D[24], fma((-M[3]), D[18], fma((-M[2]), D[17], fma((-M[1]), D[14], M[0] * D[8]))))))))));
  red(8, 2, fma((M[9] * T(0.5)), D[34], fma(M[8], D[33], fma((M[7] * T(0.5)), D[32], fma(M[6], D[29], fma(M[5], D[28], fma((M[4] * T(0.5)), D[25], fma((-M[3]), D[19], fma((-M[2]), D[18], fma((-M[1]), D[15], M[0] * D[9]))))))))));
  red(9, 3, fma((-M[3]), D[22], fma((-M[2]), D[21], fma((-M[1]), D[20], M[0] * D[10]))));
  red(10, 3, fma((-M[3]), D[24], fma((-M[2]), D[23], fma((-M[1]), D[21], M[0] * D[11]))));
  red(11, 3, fma((-M[3]), D[25], fma((-M[2]), D[24], fma((-M[1]), D[22], M[0] * D[12]))));
  red(12, 3, fma((-M[3]), D[27], fma((-M[2]), D[26], fma((-M[1]), D[23], M[0] * D[13]))));
  red(13, 3, fma((-M[3]), D[28], fma((-M[2]), D[27], fma((-M[1]), D[24], M[0] * D[14]))));
  red(14, 3, fma((-M[3]), D[29], fma((-M[2]), D[28], fma((-M[1]), D[25], M[0] * D[15]))));
  red(15, 3, fma((-M[3]), D[31], fma((-M[2]), D[30], fma((-M[1]), D[26], M[0] * D[16]))));
  red(16, 3, fma((-M[3]), D[32], fma((-M[2]), D[31], fma((-M[1]), D[27], M[0] * D[17]))));
  red(17, 3, fma((-M[3]), D[33], fma((-M[2]), D[32], fma((-M[1]), D[28], M[0] * D[18]))));
  red(18, 3, fma((-M[3]), D[34], fma((-M[2]), D[33], fma((-M[1]), D[29], M[0] * D[19]))));
  red(19, 4, M[0] * D[20]);
  red(20, 4, M[0] * D[21]);
  red(21, 4, M[0] * D[22]);
  red(22, 4, M[0] * D[23]);
  red(23, 4, M[0] * D[24]);
  red(24, 4, M[0] * D[25]);
  red(25, 4, M[0] * D[26]);
  red(26, 4, M[0] * D[27]);
  red(27, 4, M[0] * D[28]);
  red(28, 4, M[0] * D[29]);
  red(29, 4, M[0] * D[30]);
  red(30, 4, M[0] * D[31]);
  red(31, 4, M[0] * D[32]);
  red(32, 4, M[0] * D[33]);
  red(33, 4, M[0] * D[34]);
}

template <typename T>
__device__ __forceinline__ void dtensor_p5(T Rx, T Ry, T Rz, T eps2, T* __restrict__ D) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T g0_0 = nbody_rsqrt(s);
  const T is = g0_0 * g0_0;
  const T g1_0 = g0_0 * (T(-1) * is);
  const T g2_0 = g1_0 * (T(-3) * is);
  const T g3_0 = g2_0 * (T(-5) * is);
  const T g4_0 = g3_0 * (T(-7) * is);
  const T g5_0 = g4_0 * (T(-9) * is);
  const T g0_1 = Rx * g1_0;
  const T g1_1 = Rx * g2_0;
  const T g2_1 = Rx * g3_0;
  const T g3_1 = Rx * g4_0;
  const T g4_1 = Rx * g5_0;
  const T g0_2 = Ry * g1_0;
  const T g1_2 = Ry * g2_0;
  const T g2_2 = Ry * g3_0;
  const T g3_2 = Ry * g4_0;
  const T g4_2 = Ry * g5_0;
  const T g0_3 = Rz * g1_0;
  const T g1_3 = Rz * g2_0;
  const T g2_3 = Rz * g3_0;
  const T g3_3 = Rz * g4_0;
  const T g4_3 = Rz * g5_0;
  const T g0_4 = fma(T(1), g1_0, Rx * g1_1);
  const T g1_4 = fma(T(1), g2_0, Rx * g2_1);
  const T g2_4 = fma(T(1), g3_0, Rx * g3_1);
  const T g3_4 = fma(T(1), g4_0, Rx * g4_1);
  const T g0_5 = Rx * g1_2;
  const T g1_5 = Rx * g2_2;
  const T g2_5 = Rx * g3_2;
  const T g3_5 = Rx * g4_2;
  const T g0_6 = Rx * g1_3;
  const T g1_6 = Rx * g2_3;
  const T g2_6 = Rx * g3_3;
  const T g3_6 = Rx * g4_3;
  const T g0_7 = fma(T(1), g1_0, Ry * g1_2);
  const T g1_7 = fma(T(1), g2_0, Ry * g2_2);
  const T g2_7 = fma(T(1), g3_0, Ry * g3_2);
  const T g3_7 = fma(T(1), g4_0, Ry * g4_2);
  const T g0_8 = Ry * g1_3;
  const T g1_8 = Ry * g2_3;
  const T g2_8 = Ry * g3_3;
  const T g3_8 = Ry * g4_3;
  const T g0_9 = fma(T(1), g1_0, Rz * g1_3);
  const T g1_9 = fma(T(1), g2_0, Rz * g2_3);
  const T g2_9 = fma(T(1), g3_0, Rz * g3_3);
  const T g3_9 = fma(T(1), g4_0, Rz * g4_3);
  const T g0_10 = fma(T(2), g1_1, Rx * g1_4);
  const T g1_10 = fma(T(2), g2_1, Rx * g2_4);
  const T g2_10 = fma(T(2), g3_1, Rx * g3_4);
  const T g0_11 = fma(T(1), g1_2, Rx * g1_5);
  const T g1_11 = fma(T(1), g2_2, Rx * g2_5);
  const T g2_11 = fma(T(1), g3_2, Rx * g3_5);
  const T g0_12 = fma(T(1), g1_3, Rx * g1_6);
  const T g1_12 = fma(T(1), g2_3, Rx * g2_6);
  const T g2_12 = fma(T(1), g3_3, Rx * g3_6);
  const T g0_13 = Rx * g1_7;
  const T g1_13 = Rx * g2_7;
  const T g2_13 = Rx * g3_7;
  const T g0_14 = Rx * g1_8;
  const T g1_14 = Rx * g2_8;
  const T g2_14 = Rx * g3_8;
  const T g0_15 = Rx * g1_9;
  const T g1_15 = Rx * g2_9;
  const T g2_15 = Rx * g3_9;
  const T g0_16 = fma(T(2), g1_2, Ry * g1_7);
  const T g1_16 = fma(T(2), g2_2, Ry * g2_7);
  const T g2_16 = fma(T(2), g3_2, Ry * g3_7);
  const T g0_17 = fma(T(1), g1_3, Ry * g1_8);
  const T g1_17 = fma(T(1), g2_3, Ry * g2_8);
  const T g2_17 = fma(T(1), g3_3, Ry * g3_8);
  const T g0_18 = Ry * g1_9;
  const T g1_18 = Ry * g2_9;
  const T g2_18 = Ry * g3_9;
  const T g0_19 = fma(T(2), g1_3, Rz * g1_9);
  const T g1_19 = fma(T(2), g2_3, Rz * g2_9);
  const T g2_19 = fma(T(2), g3_3, Rz * g3_9);
  const T g0_20 = fma(T(3), g1_4, Rx * g1_10);
  const T g1_20 = fma(T(3), g2_4, Rx * g2_10);
  const T g0_21 = fma(T(2), g1_5, Rx * g1_11);
  const T g1_21 = fma(T(2), g2_5, Rx * g2_11);
  const T g0_22 = fma(T(2), g1_6, Rx * g1_12);
  const T g1_22 = fma(T(2), g2_6, Rx * g2_12);
  const T g0_23 = fma(T(1), g1_7, Rx * g1_13);
  const T g1_23 = fma(T(1), g2_7, Rx * g2_13);
  const T g0_24 = fma(T(1), g1_8, Rx * g1_14);
  const T g1_24 = fma(T(1), g2_8, Rx * g2_14);
  const T g0_25 = fma(T(1), g1_9, Rx * g1_15);
  const T g1_25 = fma(T(1), g2_9, Rx * g2_15);
  const T g0_26 = Rx * g1_16;
  const T g1_26 = Rx * g2_16;
  const T g0_27 = Rx * g1_17;
  const T g1_27 = Rx * g2_17;
  const T g0_28 = Rx * g1_18;
  const T g1_28 = Rx * g2_18;
  const T g0_29 = Rx * g1_19;
  const T g1_29 = Rx * g2_19;
  const T g0_30 = fma(T(3), g1_7, Ry * g1_16);
  const T g1_30 = fma(T(3), g2_7, Ry * g2_16);
  const T g0_31 = fma(T(2), g1_8, Ry * g1_17);
  const T g1_31 = fma(T(2), g2_8, Ry * g2_17);
  const T g0_32 = fma(T(1), g1_9, Ry * g1_18);
  const T g1_32 = fma(T(1), g2_9, Ry * g2_18);
  const T g0_33 = Ry * g1_19;
  const T g1_33 = Ry * g2_19;
  const T g0_34 = fma(T(3), g1_9, Rz * g1_19);
  const T g1_34 = fma(T(3), g2_9, Rz * g2_19);
  const T g0_35 = fma(T(4), g1_10, Rx * g1_20);
  const T g0_36 = fma(T(3), g1_11, Rx * g1_21);
  const T g0_37 = fma(T(3), g1_12, Rx * g1_22);
  const T g0_38 = fma(T(2), g1_13, Rx * g1_23);
  const T g0_39 = fma(T(2), g1_14, Rx * g1_24);
  const T g0_40 = fma(T(2), g1_15, Rx * g1_25);
  const T g0_41 = fma(T(1), g1_16, Rx * g1_26);
  const T g0_42 = fma(T(1), g1_17, Rx * g1_27);
  const T g0_43 = fma(T(1), g1_18, Rx * g1_28);
  const T g0_44 = fma(T(1), g1_19, Rx * g1_29);
  const T g0_45 = Rx * g1_30;
  const T g0_46 = Rx * g1_31;
  const T g0_47 = Rx * g1_32;
  const T g0_48 = Rx * g1_33;
  const T g0_49 = Rx * g1_34;
  const T g0_50 = fma(T(4), g1_16, Ry * g1_30);
  const T g0_51 = fma(T(3), g1_17, Ry * g1_31);
  const T g0_52 = fma(T(2), g1_18, Ry * g1_32);
  const T g0_53 = fma(T(1), g1_19, Ry * g1_33);
  const T g0_54 = Ry * g1_34;
  const T g0_55 = fma(T(4), g1_19, Rz * g1_34);
  D[0] = g0_0;
  D[1] = g0_1;
  D[2] = g0_2;
  D[3] = g0_3;
  D[4] = g0_4;
  D[5] = g0_5;
  D[6] = g0_6;
  D[7] = g0_7;
  D[8] = g0_8;
  D[9] = g0_9;
  D[10] = g0_10;
  D[11] = g0_11;
  D[12] = g0_12;
  D[13] = g0_13;
  D[14] = g0_14;
  D[15] = g0_15;
  D[16] = g0_16;
  D[17] = g0_17;
  D[18] = g0_18;
  D[19] = g0_19;
  D[20] = g0_20;
  D[21] = g0_21;
  D[22] = g0_22;
  D[23] = g0_23;
  D[24] = g0_24;
  D[25] = g0_25;
  D[26] = g0_26;
  D[27] = g0_27;
  D[28] = g0_28;
  D[29] = g0_29;
  D[30] = g0_30;
  D[31] = g0_31;
  D[32] = g0_32;
  D[33] = g0_33;
  D[34] = g0_34;
  D[35] = g0_35;
  D[36] = g0_36;
  D[37] = g0_37;
  D[38] = g0_38;
  D[39] = g0_39;
  D[40] = g0_40;
  D[41] = g0_41;
  D[42] = g0_42;
  D[43] = g0_43;
  D[44] = g0_44;
  D[45] = g0_45;
  D[46] = g0_46;
  D[47] = g0_47;
  D[48] = g0_48;
  D[49] = g0_49;
  D[50] = g0_50;
  D[51] = g0_51;
  D[52] = g0_52;
  D[53] = g0_53;
  D[54] = g0_54;
  D[55] = g0_55;
}

template <typename T, typename MA, typename Red>
__device__ __forceinline__ void m2l_red_p4(const MA& M, const T* __restrict__ D, Red&& red) {
  red(0, 1, fma((M[34] * T(0.041666666666666664)), D[49], fma((M[33] * T(0.16666666666666666)), D[48], fma((M[32] * T(0.25)), D[47], fma((M[31] * T(0.16666666666666666)), D[46], fma((M[30] * T(0.041666666666666664)), D[45], fma((M[29] * T(0.16666666666666666)), D[44], fma((M[28] * T(0.5)), D[43], fma((M[27] * T(0.5)), D[42], fma((M[26] * T(0.16666666666666666)), D[41], fma((M[25] * T(0.25)), D[40], fma((M[24] * T(0.5)), D[39], fma((M[23] * T(0.25)), D[38], fma((M[22] * T(0.16666666666666666)), D[37], fma((M[21] * T(0.16666666666666666)), D[36], fma((M[20] * T(0.041666666666666664)), D[35], fma((M[19] * T(-0.16666666666666666)), D[29], fma((M[18] * T(-0.5)), D[28], fma((M[17] * T(-0.5)), D[27], fma((M[16] * T(-0.16666666666666666)), D[26], fma((M[15] * T(-0.5)), D[25], fma((-M[14]), D[24], fma((M[13] * T(-0.5)), D[23], fma((M[12] * T(-0.5)), D[22], fma((M[11] * T(-0.5)), D[21], fma((M[10] * T(-0.16666666666666666)), D[20], fma((M[9] * T(0.5)), D[15], fma(M[8], D[14], fma((M[7] * T(0.5)), D[13], fma(M[6], D[12], fma(M[5], D[11], fma((M[4] * T(0.5)), D[10], fma((-M[3]), D[6], fma((-M[2]), D[5], fma((-M[1]), D[4], M[0] * D[1])))))))))))))))))))))))))))))))))));
  red(1, 1, fma((M[34] * T(0.041666666666666664)), D[54], fma((M[33] * T(0.16666666666666666)), D[53], fma((M[32] * T(0.25)), D[52], fma((M[31] * T(0.16666666666666666)), D[51], fma((M[30] * T(0.041666666666666664)), D[50], fma((M[29] * T(0.16666666666666666)), D[48], fma((M[28] * T(0.5)), D[47], fma((M[27] * T(0.5)), D[46], fma((M[26] * T(0.16666666666666666)), D[45], fma((M[25] * T(0.25)), D[43], fma((M[24] * T(0.5)), D[42], fma((M[23] * T(0.25)), D[41], fma((M[22] * T(0.16666666666666666)), D[39], fma((M[21] * T(0.16666666666666666)), D[38], fma((M[20] * T(0.041666666666666664)), D[36], fma((M[19] * T(-0.16666666666666666)), D[33], fma((M[18] * T(-0.5)), D[32], fma((M[17] * T(-0.5)), D[31], fma((M[16] * T(-0.16666666666666666)), D[30], fma((M[15] * T(-0.5)), D[28], fma((-M[14]), D[27], fma((M[13] * T(-0.5)), D[26], fma((M[12] * T(-0.5)), D[24], fma((M[11] * T(-0.5)), D[23], fma((M[10] * T(-0.16666666666666666)), D[21], fma((M[9] * T(0.5)), D[18], fma(M[8], D[17], fma((M[7] * T(0.5)), D[16], fma(M[6], D[14], fma(M[5], D[13], fma((M[4] * T(0.5)), D[11], fma((-M[3]), D[8], fma((-M[2]), D[7], fma((-M[1]), D[5], M[0] * D[2])))))))))))))))))))))))))))))))))));
  red(2, 1, fma((M[34] * T(0.041666666666666664)), D[55], fma((M[33] * T(0.16666666666666666)), D[54], fma((M[32] * T(0.25)), D[53], fma((M[31] * T(0.16666666666666666)), D[52], fma((M[30] * T(0.041666666666666664)), D[51], fma((M[29] * T(0.16666666666666666)), D[49], fma((M[28] * T(0.5)), D[48], fma((M[27] * T(0.5)), D[47], fma((M[26] * T(0.16666666666666666)), D[46], fma((M[25] * T(0.25)), D[44], fma((M[24] * T(0.5)), D[43], fma((M[23] * T(0.25)), D[42], fma((M[22] * T(0.16666666666666666)), D[40], fma((M[21] * T(0.16666666666666666)), D[39], fma((M[20] * T(0.041666666666666664)), D[37], fma((M[19] * T(-0.16666666666666666)), D[34], fma((M[18] * T(-0.5)), D[33], fma((M[17] * T(-0.5)), D[32], fma((M[16] * T(-0.16666666666666666)), D[31], fma((M[15] * T(-0.5)), D[29], fma((-M[14]), D[28], fma((M[13] * T(-0.5)), D[27], fma((M[12] * T(-0.5)), D[25], fma((M[11] * T(-0.5)), D[24], fma((M[10] * T(-0.16666666666666666)), D[22], fma((M[9] * T(0.5)), D[19], fma(M[8], D[18], fma((M[7] * T(0.5)), D[17], fma(M[6], D[15], fma(M[5], D[14], fma((M[4] * T(0.5)), D[12], fma((-M[3]), D[9], fma((-M[2]), D[8], fma((-M[1]), D[6], M[0] * D[3])))))))))))))))))))))))))))))))))));
  red(3, 2, fma((M[19] * T(-0.16666666666666666)), D[44], fma((M[18] * T(-0.5)), D[43], fma((M[17] * T(-0.5)), D[42], fma((M[16] * T(-0.16666666666666666)), D[41], fma((M[15] * T(-0.5)), D[40], fma((-M[14]), D[39], fma((M[13] * T(-0.5)), D[38], fma((M[12] * T(-0.5)), D[37], fma((M[11] * T(-0.5)), D[36], fma((M[10] * T(-0.16666666666666666)), D[35], fma((M[9] * T(0.5)), D[25], fma(M[8], D[24], fma((M[7] * T(0.5)), D[23], fma(M[6], D[22], fma(M[5], D[21], fma((M[4] * T(0.5)), D[20], fma((-M[3]), D[12], fma((-M[2]), D[11], fma((-M[1]), D[10], M[0] * D[4]))))))))))))))))))));
  red(4, 2, fma((M[19] * T(-0.16666666666666666)), D[48], fma((M[18] * T(-0.5)), D[47], fma((M[17] * T(-0.5)), D[46], fma((M[16] * T(-0.16666666666666666)), D[45], fma((M[15] * T(-0.5)), D[43], fma((-M[14]), D[42], fma((M[13] * T(-0.5)), D[41], fma((M[12] * T(-0.5)), D[39], fma((M[11] * T(-0.5)), D[38], fma((M[10] * T(-0.16666666666666666)), D[36], fma((M[9] * T(0.5)), D[28], fma(M[8], D[27], fma((M[7] * T(0.5)), D[26], fma(M[6], D[24], fma(M[5], D[23], fma((M[4] * T(0.5)), D[21], fma((-M[3]), D[14], fma((-M[2]), D[13], fma((-M[1]), D[11], M[0] * D[5]))))))))))))))))))));
  red(5, 2, fma((M[19] * T(-0.16666666666666666)), D[49], fma((M[18] * T(-0.5)), D[48], fma((M[17] * T(-0.5)), D[47], fma((M[16] * T(-0.16666666666666666)), D[46], fma((M[15] * T(-0.5)), D[44], fma((-M[14]), D[43], fma((M[13] * T(-0.5)), D[42], fma((M[12] * T(-0.5)), D[40], fma((M[11] * T(-0.5)), D[39], fma((M[10] * T(-0.16666666666666666)), D[37], fma((M[9] * T(0.5)), D[29], fma(M[8], D[28], fma((M[7] * T(0.5)), D[27], fma(M[6], D[25], fma(M[5], D[24], fma((M[4] * T(0.5)), D[22], fma((-M[3]), D[15], fma((-M[2]), D[14], fma((-M[1]), D[12], M[0] * D[6]))))))))))))))))))));
  red(6, 2, fma((M[19] * T(-0.16666666666666666)), D[53], fma((M[18] * T(-0.5)), D[52], fma((M[17] * T(-0.5)), D[51], fma((M[16] * T(-0.16666666666666666)), D[50], fma((M[15] * T(-0.5)), D[47], fma((-M[14]), D[46], fma((M[13] * T(-0.5)), D[45], fma((M[12] * T(-0.5)), D[42], fma((M[11] * T(-0.5)), D[41], fma((M[10] * T(-0.16666666666666666)), D[38], fma((M[9] * T(0.5)), D[32], fma(M[8], D[31], fma((M[7] * T(0.5)), D[30], fma(M[6], D[27], fma(M[5], D[26], fma((M[4] * T(0.5)), D[23], fma((-M[3]), D[17], fma((-M[2]), D[16], fma((-M[1]), D[13], M[0] * D[7]))))))))))))))))))));
  red(7, 2, fma((M[19] * T(-0.16666666666666666)), D[54], fma((M[18] * T(-0.5)), D[53], fma((M[17] * T(-0.5)), D[52], fma((M[16] * T(-0.16666666666666666)), D[51], fma((M[15] * T(-0.5)), D[48], fma((-M[14]), D[47], fma((M[13] * T(-0.5)), D[46], fma((M[12] * T(-0.5)), D[43], fma((M[11] * T(-0.5)), D[42], fma((M[10] * T(-0.16666666666666666)), D[39], fma((M[9] * T(0.5)), D[33], fma(M[8], D[32], fma((M[7] * T(0.5)), D[31], fma(M[6], D[28], fma(M[5], D[27], fma((M[4] * T(0.5)), D[24], fma((-M[3]), D[18], fma((-M[2]), D[17], fma((-M[1]), D[14], M[0] * D[8]))))))))))))))))))));
  red(8, 2, fma((M[19] * T(-0.16666666666666666)), D[55], fma((M[18] * T(-0.5)), D[54], fma((M[17] * T(-0.5)), D[53], fma((M[16] * T(-0.16666666666666666)), D[52], fma((M[15] * T(-0.5)), D[49], fma((-M[14]), D[48], fma((M[13] * T(-0.5)), D[47], fma((M[12] * T(-0.5)), D[44], fma((M[11] * T(-0.5)), D[43], fma((M[10] * T(-0.16666666666666666)), D[40], fma((M[9] * T(0.5)), D[34], fma(M[8], D[33], fma((M[7] * T(0.5)), D[32], fma(M[6], D[29], fma(M[5], D[28], fma((M[4] * T(0.5)), D[25], fma((-M[3]), D[19], fma((-M[2]), D[18], fma((-M[1]), D[15], M[0] * D[9]))))))))))))))))))));
  red(9, 3, fma((M[9] * T(0.5)), D[40], fma(M[8], D[39], fma((M[7] * T(0.5)), D[38], fma(M[6], D[37], fma(M[5], D[36], fma((M[4] * T(0.5)), D[35], fma((-M[3]), D[22], fma((-M[2]), D[21], fma((-M[1]), D[20], M[0] * D[10]))))))))));
  red(10, 3, fma((M[9] * T(0.5)), D[43], fma(M[8], D[42], fma((M[7] * T(0.5)), D[41], fma(M[6], D[39], fma(M[5], D[38], fma((M[4] * T(0.5)), D[36], fma((-M[3]), D[24], fma((-M[2]), D[23], fma((-M[1]), D[21], M[0] * D[11]))))))))));
  red(11, 3, fma((M[9] * T(0.5)), D[44], fma(M[8], D[43], fma((M[7] * T(0.5)), D[42], fma(M[6], D[40], fma(M[5], D[39], fma((M[4] * T(0.5)), D[37], fma((-M[3]), D[25], fma((-M[2]), D[24], fma((-M[1]), D[22], M[0] * D[12]))))))))));
  red(12, 3, fma((M[9] * T(0.5)), D[47], fma(M[8], D[46], fma((M[7] * T(0.5)), D[45], fma(M[6], D[42], fma(M[5], D[41], fma((M[4] * T(0.5)), D[38], fma((-M[3]), D[27], fma((-M[2]), D[26], fma((-M[1]), D[23], M[0] * D[13]))))))))));
  red(13, 3, fma((M[9] * T(0.5)), D[48], fma(M[8], D[47], fma((M[7] * T(0.5)), D[46], fma(M[6], D[43], fma(M[5], D[42], fma((M[4] * T(0.5)), D[39], fma((-M[3]), D[28], fma((-M[2]), D[27], fma((-M[1]), D[24], M[0] * D[14]))))))))));
  red(14, 3, fma((M[9] * T(0.5)), D[49], fma(M[8], D[48], fma((M[7] * T(0.5)), D[47], fma(M[6], D[44], fma(M[5], D[43], fma((M[4] * T(0.5)), D[40], fma((-M[3]), D[29], fma((-M[2]), D[28], fma((-M[1]), D[25], M[0] * D[15]))))))))));
  red(15, 3, fma((M[9] * T(0.5)), D[52], fma(M[8], D[51], fma((M[7] * T(0.5)), D[50], fma(M[6], D[46], fma(M[5], D[45], fma((M[4] * T(0.5)), D[41], fma((-M[3]), D[31], fma((-M[2]), D[30], fma((-M[1]), D[26], M[0] * D[16]))))))))));
  red(16, 3, fma((M[9] * T(0.5)), D[53], fma(M[8], D[52], fma((M[7] * T(0.5)), D[51], fma(M[6], D[47], fma(M[5], D[46], fma((M[4] * T(0.5)), D[42], fma((-M[3]), D[32], fma((-M[2]), D[31], fma((-M[1]), D[27], M[0] * D[17]))))))))));
  red(17, 3, fma((M[9] * T(0.5)), D[54], fma(M[8], D[53], fma((M[7] * T(0.5)), D[52], fma(M[6], D[48], fma(M[5], D[47], fma((M[4] * T(0.5)), D[43], fma((-M[3]), D[33], fma((-M[2]), D[32], fma((-M[1]), D[28], M[0] * D[18]))))))))));
  red(18, 3, fma((M[9] * T(0.5)), D[55], fma(M[8], D[54], fma((M[7] * T(0.5)), D[53], fma(M[6], D[49], fma(M[5], D[48], fma((M[4] * T(0.5)), D[44], fma((-M[3]), D[34], fma((-M[2]), D[33], fma((-M[1]), D[29], M[0] * D[19]))))))))));
  red(19, 4, fma((-M[3]), D[37], fma((-M[2]), D[36], fma((-M[1]), D[35], M[0] * D[20]))));
  red(20, 4, fma((-M[3]), D[39], fma((-M[2]), D[38], fma((-M[1]), D[36], M[0] * D[21]))));
  red(21, 4, fma((-M[3]), D[40], fma((-M[2]), D[39], fma((-M[1]), D[37], M[0] * D[22]))));
  red(22, 4, fma((-M[3]), D[42], fma((-M[2]), D[41], fma((-M[1]), D[38], M[0] * D[23]))));
  red(23, 4, fma((-M[3]), D[43], fma((-M[2]), D[42], fma((-M[1]), D[39], M[0] * D[24]))));
  red(24, 4, fma((-M[3]), D[44], fma((-M[2]), D[43], fma((-M[1]), D[40], M[0] * D[25]))));
  red(25, 4, fma((-M[3]), D[46], fma((-M[2]), D[45], fma((-M[1]), D[41], M[0] * D[26]))));
  red(26, 4, fma((-M[3]), D[47], fma((-M[2]), D[46], fma((-M[1]), D[42], M[0] * D[27]))));
  red(27, 4, fma((-M[3]), D[48], fma((-M[2]), D[47], fma((-M[1]), D[43], M[0] * D[28]))));
  red(28, 4, fma((-M[3]), D[49], fma((-M[2]), D[48], fma((-M[1]), D[44], M[0] * D[29]))));
  red(29, 4, fma((-M[3]), D[51], fma((-M[2]), D[50], fma((-M[1]), D[45], M[0] * D[30]))));
  red(30, 4, fma((-M[3]), D[52], fma((-M[2]), D[51], fma((-M[1]), D[46], M[0] * D[31]))));
  red(31, 4, fma((-M[3]), D[53], fma((-M[2]), D[52], fma((-M[1]), D[47], M[0] * D[32]))));
  red(32, 4, fma((-M[3]), D[54], fma((-M[2]), D[53], fma((-M[1]), D[48], M[0] * D[33]))));
  red(33, 4, fma((-M[3]), D[55], fma((-M[2]), D[54], fma((-M[1]), D[49], M[0] * D[34]))));
  red(34, 5, M[0] * D[35]);
  red(35, 5, M[0] * D[36]);
  red(36, 5, M[0] * D[37]);
  red(37, 5, M[0] * D[38]);
  red(38, 5, M[0] * D[39]);
  red(39, 5, M[0] * D[40]);
  red(40, 5, M[0] * D[41]);
  red(41, 5, M[0] * D[42]);
  red(42, 5, M[0] * D[43]);
  red(43, 5, M[0] * D[44]);
  red(44, 5, M[0] * D[45]);
  red(45, 5, M[0] * D[46]);
  red(46, 5, M[0] * D[47]);
  red(47, 5, M[0] * D[48]);
  red(48, 5, M[0] * D[49]);
  red(49, 5, M[0] * D[50]);
  red(50, 5, M[0] * D[51]);
  red(51, 5, M[0] * D[52]);
  red(52, 5, M[0] * D[53]);
  red(53, 5, M[0] * D[54]);
  red(54, 5, M[0] * D[55]);
}

__device__ __forceinline__ float2 nbody_rsqrt2(float2 s) {
  return make_float2(nbody_rsqrt(s.x), nbody_rsqrt(s.y));
}

template <typename T>
__device__ __forceinline__ void cube_bg_l4(T q, T Rx, T Ry, T Rz, T& ax, T& ay, T& az) {
  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;
  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));
  const T ir = nbody_rsqrt(r2);
  const T ir2 = ir * ir;
  const T u = q * ir * ir2 * ir2 * ir2 * ir2 * ir2;
  const T X0Y0Z2 = Z * Z;
  const T X0Y1Z1 = Z * Y;
  const T X0Y2Z0 = Y * Y;
  const T X1Y0Z1 = Z * X;
  const T X1Y1Z0 = Y * X;
  const T X2Y0Z0 = X * X;
  T w0 = T(0.21875) * X0Y0Z2;
  w0 = fma(T(-0.21875), X0Y1Z1, w0);
  w0 = fma(T(0.21875), X0Y2Z0, w0);
  w0 = fma(T(-0.36458333333333331), X1Y0Z1, w0);
  w0 = fma(T(-0.36458333333333331), X1Y1Z0, w0);
  w0 = fma(T(0.072916666666666671), X2Y0Z0, w0);
  T w1 = T(0.21875) * X0Y0Z2;
  w1 = fma(T(-0.36458333333333331), X0Y1Z1, w1);
  w1 = fma(T(0.072916666666666671), X0Y2Z0, w1);
  w1 = fma(T(-0.21875), X1Y0Z1, w1);
  w1 = fma(T(-0.36458333333333331), X1Y1Z0, w1);
  w1 = fma(T(0.21875), X2Y0Z0, w1);
  T w2 = T(0.072916666666666671) * X0Y0Z2;
  w2 = fma(T(-0.36458333333333331), X0Y1Z1, w2);
  w2 = fma(T(0.21875), X0Y2Z0, w2);
  w2 = fma(T(-0.36458333333333331), X1Y0Z1, w2);
  w2 = fma(T(-0.21875), X1Y1Z0, w2);
  w2 = fma(T(0.21875), X2Y0Z0, w2);
  ax = fma(Rx * u, w0, ax);
  ay = fma(Ry * u, w1, ay);
  az = fma(Rz * u, w2, az);
}

template <typename T>
__device__ __forceinline__ T cube_bgpot_l4(T q, T Rx, T Ry, T Rz) {
  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;
  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));
  const T ir = nbody_rsqrt(r2);
  const T ir2 = ir * ir;
  const T X0Y0Z2 = Z * Z;
  const T X0Y1Z1 = Z * Y;
  const T X0Y2Z0 = Y * Y;
  const T X1Y0Z1 = Z * X;
  const T X1Y1Z0 = Y * X;
  const T X2Y0Z0 = X * X;
  T hv = T(-0.014583333333333334) * X0Y0Z2;
  hv = fma(T(0.043749999999999997), X0Y1Z1, hv);
  hv = fma(T(-0.014583333333333334), X0Y2Z0, hv);
  hv = fma(T(0.043749999999999997), X1Y0Z1, hv);
  hv = fma(T(0.043749999999999997), X1Y1Z0, hv);
  hv = fma(T(-0.014583333333333334), X2Y0Z0, hv);
  return q * hv * (ir * ir2 * ir2 * ir2 * ir2);
}

__device__ __forceinline__ void cube_bg2_l4(float2 q, float2 Rx, float2 Ry, float2 Rz, float2& ax, float2& ay, float2& az) {
  const float2 X = __fmul2_rn(Rx, Rx), Y = __fmul2_rn(Ry, Ry), Z = __fmul2_rn(Rz, Rz);
  const float2 r2 = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, Z));
  const float2 ir = nbody_rsqrt2(r2);
  const float2 ir2 = __fmul2_rn(ir, ir);
  const float2 u = __fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(q, ir), ir2), ir2), ir2), ir2), ir2);
  const float2 X0Y0Z2 = __fmul2_rn(Z, Z);
  const float2 X0Y1Z1 = __fmul2_rn(Z, Y);
  const float2 X0Y2Z0 = __fmul2_rn(Y, Y);
  const float2 X1Y0Z1 = __fmul2_rn(Z, X);
  const float2 X1Y1Z0 = __fmul2_rn(Y, X);
  const float2 X2Y0Z0 = __fmul2_rn(X, X);
  float2 w0 = __fmul2_rn(make_float2(0.21875f, 0.21875f), X0Y0Z2);
  w0 = __ffma2_rn(make_float2(-0.21875f, -0.21875f), X0Y1Z1, w0);
  w0 = __ffma2_rn(make_float2(0.21875f, 0.21875f), X0Y2Z0, w0);
  w0 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X1Y0Z1, w0);
  w0 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X1Y1Z0, w0);
  w0 = __ffma2_rn(make_float2(0.0729166667f, 0.0729166667f), X2Y0Z0, w0);
  float2 w1 = __fmul2_rn(make_float2(0.21875f, 0.21875f), X0Y0Z2);
  w1 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X0Y1Z1, w1);
  w1 = __ffma2_rn(make_float2(0.0729166667f, 0.0729166667f), X0Y2Z0, w1);
  w1 = __ffma2_rn(make_float2(-0.21875f, -0.21875f), X1Y0Z1, w1);
  w1 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X1Y1Z0, w1);
  w1 = __ffma2_rn(make_float2(0.21875f, 0.21875f), X2Y0Z0, w1);
  float2 w2 = __fmul2_rn(make_float2(0.0729166667f, 0.0729166667f), X0Y0Z2);
  w2 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X0Y1Z1, w2);
  w2 = __ffma2_rn(make_float2(0.21875f, 0.21875f), X0Y2Z0, w2);
  w2 = __ffma2_rn(make_float2(-0.364583333f, -0.364583333f), X1Y0Z1, w2);
  w2 = __ffma2_rn(make_float2(-0.21875f, -0.21875f), X1Y1Z0, w2);
  w2 = __ffma2_rn(make_float2(0.21875f, 0.21875f), X2Y0Z0, w2);
  ax = __ffma2_rn(__fmul2_rn(Rx, u), w0, ax);
  ay = __ffma2_rn(__fmul2_rn(Ry, u), w1, ay);
  az = __ffma2_rn(__fmul2_rn(Rz, u), w2, az);
}

template <typename T>
__device__ __forceinline__ void cube_bg_l6(T q, T Rx, T Ry, T Rz, T& ax, T& ay, T& az) {
  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;
  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));
  const T ir = nbody_rsqrt(r2);
  const T ir2 = ir * ir;
  const T u = q * ir * ir2 * ir2 * ir2 * ir2 * ir2 * ir2 * ir2;
  const T X0Y0Z2 = Z * Z;
  const T X0Y1Z1 = Z * Y;
  const T X0Y2Z0 = Y * Y;
  const T X1Y0Z1 = Z * X;
  const T X1Y1Z0 = Y * X;
  const T X2Y0Z0 = X * X;
  const T X0Y0Z3 = X0Y0Z2 * Z;
  const T X0Y1Z2 = X0Y0Z2 * Y;
  const T X0Y2Z1 = X0Y1Z1 * Y;
  const T X0Y3Z0 = X0Y2Z0 * Y;
  const T X1Y0Z2 = X0Y0Z2 * X;
  const T X1Y1Z1 = X0Y1Z1 * X;
  const T X1Y2Z0 = X0Y2Z0 * X;
  const T X2Y0Z1 = X1Y0Z1 * X;
  const T X2Y1Z0 = X1Y1Z0 * X;
  const T X3Y0Z0 = X2Y0Z0 * X;
  T w0 = T(-0.041666666666666664) * X0Y0Z3;
  w0 = fma(T(0.390625), X0Y1Z2, w0);
  w0 = fma(T(0.390625), X0Y2Z1, w0);
  w0 = fma(T(-0.041666666666666664), X0Y3Z0, w0);
  w0 = fma(T(0.078125), X1Y0Z2, w0);
  w0 = fma(T(-1.5625), X1Y1Z1, w0);
  w0 = fma(T(0.078125), X1Y2Z0, w0);
  w0 = fma(T(0.109375), X2Y0Z1, w0);
  w0 = fma(T(0.109375), X2Y1Z0, w0);
  w0 = fma(T(-0.010416666666666666), X3Y0Z0, w0);
  T w1 = T(-0.041666666666666664) * X0Y0Z3;
  w1 = fma(T(0.078125), X0Y1Z2, w1);
  w1 = fma(T(0.109375), X0Y2Z1, w1);
  w1 = fma(T(-0.010416666666666666), X0Y3Z0, w1);
  w1 = fma(T(0.390625), X1Y0Z2, w1);
  w1 = fma(T(-1.5625), X1Y1Z1, w1);
  w1 = fma(T(0.109375), X1Y2Z0, w1);
  w1 = fma(T(0.390625), X2Y0Z1, w1);
  w1 = fma(T(0.078125), X2Y1Z0, w1);
  w1 = fma(T(-0.041666666666666664), X3Y0Z0, w1);
  T w2 = T(-0.010416666666666666) * X0Y0Z3;
  w2 = fma(T(0.109375), X0Y1Z2, w2);
  w2 = fma(T(0.078125), X0Y2Z1, w2);
  w2 = fma(T(-0.041666666666666664), X0Y3Z0, w2);
  w2 = fma(T(0.109375), X1Y0Z2, w2);
  w2 = fma(T(-1.5625), X1Y1Z1, w2);
  w2 = fma(T(0.390625), X1Y2Z0, w2);
  w2 = fma(T(0.078125), X2Y0Z1, w2);
  w2 = fma(T(0.390625), X2Y1Z0, w2);
  w2 = fma(T(-0.041666666666666664), X3Y0Z0, w2);
  ax = fma(Rx * u, w0, ax);
  ay = fma(Ry * u, w1, ay);
  az = fma(Rz * u, w2, az);
}

template <typename T>
__device__ __forceinline__ T cube_bgpot_l6(T q, T Rx, T Ry, T Rz) {
  const T X = Rx * Rx, Y = Ry * Ry, Z = Rz * Rz;
  const T r2 = fma(Rx, Rx, fma(Ry, Ry, Z));
  const T ir = nbody_rsqrt(r2);
  const T ir2 = ir * ir;
  const T X0Y0Z2 = Z * Z;
  const T X0Y1Z1 = Z * Y;
  const T X0Y2Z0 = Y * Y;
  const T X1Y0Z1 = Z * X;
  const T X1Y1Z0 = Y * X;
  const T X2Y0Z0 = X * X;
  const T X0Y0Z3 = X0Y0Z2 * Z;
  const T X0Y1Z2 = X0Y0Z2 * Y;
  const T X0Y2Z1 = X0Y1Z1 * Y;
  const T X0Y3Z0 = X0Y2Z0 * Y;
  const T X1Y0Z2 = X0Y0Z2 * X;
  const T X1Y1Z1 = X0Y1Z1 * X;
  const T X1Y2Z0 = X0Y2Z0 * X;
  const T X2Y0Z1 = X1Y0Z1 * X;
  const T X2Y1Z0 = X1Y1Z0 * X;
  const T X3Y0Z0 = X2Y0Z0 * X;
  T hv = T(0.001488095238095238) * X0Y0Z3;
  hv = fma(T(-0.011160714285714286), X0Y1Z2, hv);
  hv = fma(T(-0.011160714285714286), X0Y2Z1, hv);
  hv = fma(T(0.001488095238095238), X0Y3Z0, hv);
  hv = fma(T(-0.011160714285714286), X1Y0Z2, hv);
  hv = fma(T(0.13392857142857142), X1Y1Z1, hv);
  hv = fma(T(-0.011160714285714286), X1Y2Z0, hv);
  hv = fma(T(-0.011160714285714286), X2Y0Z1, hv);
  hv = fma(T(-0.011160714285714286), X2Y1Z0, hv);
  hv = fma(T(0.001488095238095238), X3Y0Z0, hv);
  return q * hv * (ir * ir2 * ir2 * ir2 * ir2 * ir2 * ir2);
}

__device__ __forceinline__ void cube_bg2_l6(float2 q, float2 Rx, float2 Ry, float2 Rz, float2& ax, float2& ay, float2& az) {
  const float2 X = __fmul2_rn(Rx, Rx), Y = __fmul2_rn(Ry, Ry), Z = __fmul2_rn(Rz, Rz);
  const float2 r2 = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, Z));
  const float2 ir = nbody_rsqrt2(r2);
  const float2 ir2 = __fmul2_rn(ir, ir);
  const float2 u = __fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(q, ir), ir2), ir2), ir2), ir2), ir2), ir2), ir2);
  const float2 X0Y0Z2 = __fmul2_rn(Z, Z);
  const float2 X0Y1Z1 = __fmul2_rn(Z, Y);
  const float2 X0Y2Z0 = __fmul2_rn(Y, Y);
  const float2 X1Y0Z1 = __fmul2_rn(Z, X);
  const float2 X1Y1Z0 = __fmul2_rn(Y, X);
  const float2 X2Y0Z0 = __fmul2_rn(X, X);
  const float2 X0Y0Z3 = __fmul2_rn(X0Y0Z2, Z);
  const float2 X0Y1Z2 = __fmul2_rn(X0Y0Z2, Y);
  const float2 X0Y2Z1 = __fmul2_rn(X0Y1Z1, Y);
  const float2 X0Y3Z0 = __fmul2_rn(X0Y2Z0, Y);
  const float2 X1Y0Z2 = __fmul2_rn(X0Y0Z2, X);
  const float2 X1Y1Z1 = __fmul2_rn(X0Y1Z1, X);
  const float2 X1Y2Z0 = __fmul2_rn(X0Y2Z0, X);
  const float2 X2Y0Z1 = __fmul2_rn(X1Y0Z1, X);
  const float2 X2Y1Z0 = __fmul2_rn(X1Y1Z0, X);
  const float2 X3Y0Z0 = __fmul2_rn(X2Y0Z0, X);
  float2 w0 = __fmul2_rn(make_float2(-0.0416666667f, -0.0416666667f), X0Y0Z3);
  w0 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X0Y1Z2, w0);
  w0 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X0Y2Z1, w0);
  w0 = __ffma2_rn(make_float2(-0.0416666667f, -0.0416666667f), X0Y3Z0, w0);
  w0 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X1Y0Z2, w0);
  w0 = __ffma2_rn(make_float2(-1.5625f, -1.5625f), X1Y1Z1, w0);
  w0 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X1Y2Z0, w0);
  w0 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X2Y0Z1, w0);
  w0 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X2Y1Z0, w0);
  w0 = __ffma2_rn(make_float2(-0.0104166667f, -0.0104166667f), X3Y0Z0, w0);
  float2 w1 = __fmul2_rn(make_float2(-0.0416666667f, -0.0416666667f), X0Y0Z3);
  w1 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X0Y1Z2, w1);
  w1 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X0Y2Z1, w1);
  w1 = __ffma2_rn(make_float2(-0.0104166667f, -0.0104166667f), X0Y3Z0, w1);
  w1 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X1Y0Z2, w1);
  w1 = __ffma2_rn(make_float2(-1.5625f, -1.5625f), X1Y1Z1, w1);
  w1 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X1Y2Z0, w1);
  w1 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X2Y0Z1, w1);
  w1 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X2Y1Z0, w1);
  w1 = __ffma2_rn(make_float2(-0.0416666667f, -0.0416666667f), X3Y0Z0, w1);
  float2 w2 = __fmul2_rn(make_float2(-0.0104166667f, -0.0104166667f), X0Y0Z3);
  w2 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X0Y1Z2, w2);
  w2 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X0Y2Z1, w2);
  w2 = __ffma2_rn(make_float2(-0.0416666667f, -0.0416666667f), X0Y3Z0, w2);
  w2 = __ffma2_rn(make_float2(0.109375f, 0.109375f), X1Y0Z2, w2);
  w2 = __ffma2_rn(make_float2(-1.5625f, -1.5625f), X1Y1Z1, w2);
  w2 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X1Y2Z0, w2);
  w2 = __ffma2_rn(make_float2(0.078125f, 0.078125f), X2Y0Z1, w2);
  w2 = __ffma2_rn(make_float2(0.390625f, 0.390625f), X2Y1Z0, w2);
  w2 = __ffma2_rn(make_float2(-0.0416666667f, -0.0416666667f), X3Y0Z0, w2);
  ax = __ffma2_rn(__fmul2_rn(Rx, u), w0, ax);
  ay = __ffma2_rn(__fmul2_rn(Ry, u), w1, ay);
  az = __ffma2_rn(__fmul2_rn(Rz, u), w2, az);
}

