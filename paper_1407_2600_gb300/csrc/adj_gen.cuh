// Generated by gen_m2p.py -- do not edit by hand.
// Reverse-mode (adjoint) kernels of the M2P, M2M, P2M and image-field expansions.
#pragma once

template <typename T>
__device__ __forceinline__ void cube_bg_hvp_l4(T q, T Rx, T Ry, T Rz, T lx, T ly, T lz, T& ox, T& oy,
                                             T& oz) {
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
  T d00 = T(-0.36458333333333331) * Z;
  d00 = fma(T(-0.36458333333333331), Y, d00);
  d00 = fma(T(0.14583333333333334), X, d00);
  T d01 = T(-0.21875) * Z;
  d01 = fma(T(0.4375), Y, d01);
  d01 = fma(T(-0.36458333333333331), X, d01);
  T d02 = T(0.4375) * Z;
  d02 = fma(T(-0.21875), Y, d02);
  d02 = fma(T(-0.36458333333333331), X, d02);
  T d10 = T(-0.21875) * Z;
  d10 = fma(T(-0.36458333333333331), Y, d10);
  d10 = fma(T(0.4375), X, d10);
  T d11 = T(-0.36458333333333331) * Z;
  d11 = fma(T(0.14583333333333334), Y, d11);
  d11 = fma(T(-0.36458333333333331), X, d11);
  T d12 = T(0.4375) * Z;
  d12 = fma(T(-0.36458333333333331), Y, d12);
  d12 = fma(T(-0.21875), X, d12);
  T d20 = T(-0.36458333333333331) * Z;
  d20 = fma(T(-0.21875), Y, d20);
  d20 = fma(T(0.4375), X, d20);
  T d21 = T(-0.36458333333333331) * Z;
  d21 = fma(T(0.4375), Y, d21);
  d21 = fma(T(-0.21875), X, d21);
  T d22 = T(0.14583333333333334) * Z;
  d22 = fma(T(-0.36458333333333331), Y, d22);
  d22 = fma(T(-0.36458333333333331), X, d22);
  const T t0 = T(2) * Rx * lx, t1 = T(2) * Ry * ly, t2 = T(2) * Rz * lz;
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz)) * (T(-11) * ir2);
  const T s0 = fma(d00, t0, fma(d01, t1, d02 * t2));
  ox = fma(u, fma(w0, lx, Rx * fma(w0, rl, s0)), ox);
  const T s1 = fma(d10, t0, fma(d11, t1, d12 * t2));
  oy = fma(u, fma(w1, ly, Ry * fma(w1, rl, s1)), oy);
  const T s2 = fma(d20, t0, fma(d21, t1, d22 * t2));
  oz = fma(u, fma(w2, lz, Rz * fma(w2, rl, s2)), oz);
}

template <typename T>
__device__ __forceinline__ void cube_bg_hvp_l6(T q, T Rx, T Ry, T Rz, T lx, T ly, T lz, T& ox, T& oy,
                                             T& oz) {
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
  T d00 = T(0.078125) * X0Y0Z2;
  d00 = fma(T(-1.5625), X0Y1Z1, d00);
  d00 = fma(T(0.078125), X0Y2Z0, d00);
  d00 = fma(T(0.21875), X1Y0Z1, d00);
  d00 = fma(T(0.21875), X1Y1Z0, d00);
  d00 = fma(T(-0.03125), X2Y0Z0, d00);
  T d01 = T(0.390625) * X0Y0Z2;
  d01 = fma(T(0.78125), X0Y1Z1, d01);
  d01 = fma(T(-0.125), X0Y2Z0, d01);
  d01 = fma(T(-1.5625), X1Y0Z1, d01);
  d01 = fma(T(0.15625), X1Y1Z0, d01);
  d01 = fma(T(0.109375), X2Y0Z0, d01);
  T d02 = T(-0.125) * X0Y0Z2;
  d02 = fma(T(0.78125), X0Y1Z1, d02);
  d02 = fma(T(0.390625), X0Y2Z0, d02);
  d02 = fma(T(0.15625), X1Y0Z1, d02);
  d02 = fma(T(-1.5625), X1Y1Z0, d02);
  d02 = fma(T(0.109375), X2Y0Z0, d02);
  T d10 = T(0.390625) * X0Y0Z2;
  d10 = fma(T(-1.5625), X0Y1Z1, d10);
  d10 = fma(T(0.109375), X0Y2Z0, d10);
  d10 = fma(T(0.78125), X1Y0Z1, d10);
  d10 = fma(T(0.15625), X1Y1Z0, d10);
  d10 = fma(T(-0.125), X2Y0Z0, d10);
  T d11 = T(0.078125) * X0Y0Z2;
  d11 = fma(T(0.21875), X0Y1Z1, d11);
  d11 = fma(T(-0.03125), X0Y2Z0, d11);
  d11 = fma(T(-1.5625), X1Y0Z1, d11);
  d11 = fma(T(0.21875), X1Y1Z0, d11);
  d11 = fma(T(0.078125), X2Y0Z0, d11);
  T d12 = T(-0.125) * X0Y0Z2;
  d12 = fma(T(0.15625), X0Y1Z1, d12);
  d12 = fma(T(0.109375), X0Y2Z0, d12);
  d12 = fma(T(0.78125), X1Y0Z1, d12);
  d12 = fma(T(-1.5625), X1Y1Z0, d12);
  d12 = fma(T(0.390625), X2Y0Z0, d12);
  T d20 = T(0.109375) * X0Y0Z2;
  d20 = fma(T(-1.5625), X0Y1Z1, d20);
  d20 = fma(T(0.390625), X0Y2Z0, d20);
  d20 = fma(T(0.15625), X1Y0Z1, d20);
  d20 = fma(T(0.78125), X1Y1Z0, d20);
  d20 = fma(T(-0.125), X2Y0Z0, d20);
  T d21 = T(0.109375) * X0Y0Z2;
  d21 = fma(T(0.15625), X0Y1Z1, d21);
  d21 = fma(T(-0.125), X0Y2Z0, d21);
  d21 = fma(T(-1.5625), X1Y0Z1, d21);
  d21 = fma(T(0.78125), X1Y1Z0, d21);
  d21 = fma(T(0.390625), X2Y0Z0, d21);
  T d22 = T(-0.03125) * X0Y0Z2;
  d22 = fma(T(0.21875), X0Y1Z1, d22);
  d22 = fma(T(0.078125), X0Y2Z0, d22);
  d22 = fma(T(0.21875), X1Y0Z1, d22);
  d22 = fma(T(-1.5625), X1Y1Z0, d22);
  d22 = fma(T(0.078125), X2Y0Z0, d22);
  const T t0 = T(2) * Rx * lx, t1 = T(2) * Ry * ly, t2 = T(2) * Rz * lz;
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz)) * (T(-15) * ir2);
  const T s0 = fma(d00, t0, fma(d01, t1, d02 * t2));
  ox = fma(u, fma(w0, lx, Rx * fma(w0, rl, s0)), ox);
  const T s1 = fma(d10, t0, fma(d11, t1, d12 * t2));
  oy = fma(u, fma(w1, ly, Ry * fma(w1, rl, s1)), oy);
  const T s2 = fma(d20, t0, fma(d21, t1, d22 * t2));
  oz = fma(u, fma(w2, lz, Rz * fma(w2, rl, s2)), oz);
}

template <typename T>
__device__ __forceinline__ void m2p_adj_self_p0(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T m0 = T(1);
  T S0;
  { const T b = B[0];
    S0 = b;
  }
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  T ax = ox, ay = oy, az = oz;
  { const T a1 = F1 * S0;  // F_{j+1} S_j
    const T c1 = F2 * S0 * rl;  // R_k coefficient
    ax = fma(a1, lx, fma(Rx, c1, ax));
    ay = fma(a1, ly, fma(Ry, c1, ay));
    az = fma(a1, lz, fma(Rz, c1, az));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

__device__ __forceinline__ void m2p2_adj_self_p0(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz, float2 eps2, float2 lx, float2 ly, float2 lz, float2& ox, float2& oy, float2& oz) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = nbody_rsqrt2(s);
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 m0 = make_float2(1.0f, 1.0f);
  float2 S0;
  { const float2 b = B[0];
    S0 = b;
  }
  const float2 rl = __ffma2_rn(Rx, lx, __ffma2_rn(Ry, ly, __fmul2_rn(Rz, lz)));
  float2 ax = ox, ay = oy, az = oz;
  { const float2 a1 = __fmul2_rn(F1, S0);
    const float2 c1 = __fmul2_rn(__fmul2_rn(F2, S0), rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, ax));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, ay));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, az));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

template <typename T>
__device__ __forceinline__ void m2p_adj_src_p0(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz,
                                         T* __restrict__ nu) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T r0 = T(1);
  const T E0 = F1 * (r0);
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  nu[0] = fma(rl, E0, nu[0]);
}

__device__ __forceinline__ void m2m_adj_acc_p0(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {
  const double w0 = 1.0;
  nuc[0] = fma(w0, nup[0], nuc[0]);
}

__device__ __forceinline__ void p2m_adj_p0(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {
  const double q0 = 1.0;
  gx = fma(m, 0.0, gx);
  gy = fma(m, 0.0, gy);
  gz = fma(m, 0.0, gz);
}

template <typename T>
__device__ __forceinline__ void m2p_adj_self_p1(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T m0 = T(1);
  const T m1 = Rx;
  const T m2 = Ry;
  const T m3 = Rz;
  T S0, S1, G1x, G1y, G1z;
  { const T b = B[0];
    S0 = b;
  }
  { const T b = B[1];
    S1 = b * m1;
    G1x = b;
  }
  { const T b = B[2];
    S1 = fma(b, m2, S1);
    G1y = b;
  }
  { const T b = B[3];
    S1 = fma(b, m3, S1);
    G1z = b;
  }
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  T ax = ox, ay = oy, az = oz;
  { const T a1 = F1 * S0;  // F_{j+1} S_j
    const T c1 = F2 * S0 * rl;  // R_k coefficient
    ax = fma(a1, lx, fma(Rx, c1, ax));
    ay = fma(a1, ly, fma(Ry, c1, ay));
    az = fma(a1, lz, fma(Rz, c1, az));
  }
  { const T a1 = F2 * S1;  // F_{j+1} S_j
    const T gl = fma(G1x, lx, fma(G1y, ly, G1z * lz));
    const T c1 = fma(F3 * S1, rl, F2 * gl);  // R_k coefficient
    const T c2 = F2 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G1x, ax)));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G1y, ay)));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G1z, az)));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

__device__ __forceinline__ void m2p2_adj_self_p1(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz, float2 eps2, float2 lx, float2 ly, float2 lz, float2& ox, float2& oy, float2& oz) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = nbody_rsqrt2(s);
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 m0 = make_float2(1.0f, 1.0f);
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
  const float2 rl = __ffma2_rn(Rx, lx, __ffma2_rn(Ry, ly, __fmul2_rn(Rz, lz)));
  float2 ax = ox, ay = oy, az = oz;
  { const float2 a1 = __fmul2_rn(F1, S0);
    const float2 c1 = __fmul2_rn(__fmul2_rn(F2, S0), rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, ax));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, ay));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, az));
  }
  { const float2 a1 = __fmul2_rn(F2, S1);
    const float2 gl = __ffma2_rn(G1x, lx, __ffma2_rn(G1y, ly, __fmul2_rn(G1z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F3, S1), rl, __fmul2_rn(F2, gl));
    const float2 c2 = __fmul2_rn(F2, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G1x, ax)));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G1y, ay)));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G1z, az)));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

template <typename T>
__device__ __forceinline__ void m2p_adj_src_p1(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz,
                                         T* __restrict__ nu) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T r0 = T(1);
  const T r1 = Rx;
  const T r2 = Ry;
  const T r3 = Rz;
  const T E0 = F1 * (r0);
  const T E1 = F2 * (r1);
  const T E2 = F2 * (r2);
  const T E3 = F2 * (r3);
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  nu[0] = fma(rl, E0, nu[0]);
  nu[1] = fma(lx, E0, fma(rl, E1, nu[1]));
  nu[2] = fma(ly, E0, fma(rl, E2, nu[2]));
  nu[3] = fma(lz, E0, fma(rl, E3, nu[3]));
}

__device__ __forceinline__ void m2m_adj_acc_p1(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {
  const double w0 = 1.0;
  const double w1 = w0 * sx;
  const double w2 = w0 * sy;
  const double w3 = w0 * sz;
  nuc[0] = fma(w3, nup[3], fma(w2, nup[2], fma(w1, nup[1], fma(w0, nup[0], nuc[0]))));
  nuc[1] = fma(w0, nup[1], nuc[1]);
  nuc[2] = fma(w0, nup[2], nuc[2]);
  nuc[3] = fma(w0, nup[3], nuc[3]);
}

__device__ __forceinline__ void p2m_adj_p1(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {
  const double q0 = 1.0;
  gx = fma(m, fma(nu[1], q0, 0.0), gx);
  gy = fma(m, fma(nu[2], q0, 0.0), gy);
  gz = fma(m, fma(nu[3], q0, 0.0), gz);
}

template <typename T>
__device__ __forceinline__ void m2p_adj_self_p2(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
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
  T q1 = lx;
  T q2 = ly;
  T q3 = lz;
  T S0, S1, G1x, G1y, G1z, S2, G2x, H2x, G2y, H2y, G2z, H2z;
  { const T b = B[0];
    S0 = b;
  }
  { const T b = B[1];
    S1 = b;
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = b;
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = b;
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = b;
  }
  { const T b = B[5];
    S2 = b * m4;
    G2x = b * m1;
    H2x = b * q1;
  }
  { const T b = B[6];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    H2x = fma(b, q2, H2x);
    G2y = b * m1;
    H2y = b * q1;
  }
  { const T b = B[7];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    H2x = fma(b, q3, H2x);
    G2z = b * m1;
    H2z = b * q1;
  }
  { const T b = B[8];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
    H2y = fma(b, q2, H2y);
  }
  { const T b = B[9];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    H2y = fma(b, q3, H2y);
    G2z = fma(b, m2, G2z);
    H2z = fma(b, q2, H2z);
  }
  { const T b = B[10];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
    H2z = fma(b, q3, H2z);
  }
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  T ax = ox, ay = oy, az = oz;
  { const T a1 = F1 * S0;  // F_{j+1} S_j
    const T c1 = F2 * S0 * rl;  // R_k coefficient
    ax = fma(a1, lx, fma(Rx, c1, ax));
    ay = fma(a1, ly, fma(Ry, c1, ay));
    az = fma(a1, lz, fma(Rz, c1, az));
  }
  { const T a1 = F2 * S1;  // F_{j+1} S_j
    const T gl = fma(G1x, lx, fma(G1y, ly, G1z * lz));
    const T c1 = fma(F3 * S1, rl, F2 * gl);  // R_k coefficient
    const T c2 = F2 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G1x, ax)));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G1y, ay)));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G1z, az)));
  }
  { const T a1 = F3 * S2;  // F_{j+1} S_j
    const T gl = fma(G2x, lx, fma(G2y, ly, G2z * lz));
    const T c1 = fma(F4 * S2, rl, F3 * gl);  // R_k coefficient
    const T c2 = F3 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G2x, fma(F2, H2x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G2y, fma(F2, H2y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G2z, fma(F2, H2z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

__device__ __forceinline__ void m2p2_adj_self_p2(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz, float2 eps2, float2 lx, float2 ly, float2 lz, float2& ox, float2& oy, float2& oz) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = nbody_rsqrt2(s);
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 F4 = __fmul2_rn(F3, __fmul2_rn(make_float2(-7.0f, -7.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 m0 = make_float2(1.0f, 1.0f);
  const float2 m1 = Rx;
  const float2 m2 = Ry;
  const float2 m3 = Rz;
  const float2 m4 = __fmul2_rn(m1, Rx_2);
  const float2 m5 = __fmul2_rn(m2, Rx);
  const float2 m6 = __fmul2_rn(m3, Rx);
  const float2 m7 = __fmul2_rn(m2, Ry_2);
  const float2 m8 = __fmul2_rn(m3, Ry);
  const float2 m9 = __fmul2_rn(m3, Rz_2);
  float2 q1 = lx;
  float2 q2 = ly;
  float2 q3 = lz;
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, H2x, G2y, H2y, G2z, H2z;
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
    H2x = __fmul2_rn(b, q1);
  }
  { const float2 b = B[6];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    H2x = __ffma2_rn(b, q2, H2x);
    G2y = __fmul2_rn(b, m1);
    H2y = __fmul2_rn(b, q1);
  }
  { const float2 b = B[7];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    H2x = __ffma2_rn(b, q3, H2x);
    G2z = __fmul2_rn(b, m1);
    H2z = __fmul2_rn(b, q1);
  }
  { const float2 b = B[8];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
    H2y = __ffma2_rn(b, q2, H2y);
  }
  { const float2 b = B[9];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    H2y = __ffma2_rn(b, q3, H2y);
    G2z = __ffma2_rn(b, m2, G2z);
    H2z = __ffma2_rn(b, q2, H2z);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
    H2z = __ffma2_rn(b, q3, H2z);
  }
  const float2 rl = __ffma2_rn(Rx, lx, __ffma2_rn(Ry, ly, __fmul2_rn(Rz, lz)));
  float2 ax = ox, ay = oy, az = oz;
  { const float2 a1 = __fmul2_rn(F1, S0);
    const float2 c1 = __fmul2_rn(__fmul2_rn(F2, S0), rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, ax));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, ay));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, az));
  }
  { const float2 a1 = __fmul2_rn(F2, S1);
    const float2 gl = __ffma2_rn(G1x, lx, __ffma2_rn(G1y, ly, __fmul2_rn(G1z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F3, S1), rl, __fmul2_rn(F2, gl));
    const float2 c2 = __fmul2_rn(F2, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G1x, ax)));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G1y, ay)));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G1z, az)));
  }
  { const float2 a1 = __fmul2_rn(F3, S2);
    const float2 gl = __ffma2_rn(G2x, lx, __ffma2_rn(G2y, ly, __fmul2_rn(G2z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F4, S2), rl, __fmul2_rn(F3, gl));
    const float2 c2 = __fmul2_rn(F3, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G2x, __ffma2_rn(F2, H2x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G2y, __ffma2_rn(F2, H2y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G2z, __ffma2_rn(F2, H2z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

template <typename T>
__device__ __forceinline__ void m2p_adj_src_p2(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz,
                                         T* __restrict__ nu) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T r0 = T(1);
  const T r1 = Rx;
  const T r2 = Ry;
  const T r3 = Rz;
  const T r4 = r1 * Rx;
  const T r5 = r2 * Rx;
  const T r6 = r3 * Rx;
  const T r7 = r2 * Ry;
  const T r8 = r3 * Ry;
  const T r9 = r3 * Rz;
  const T E0 = F1 * (r0);
  const T E1 = F2 * (r1);
  const T E2 = F2 * (r2);
  const T E3 = F2 * (r3);
  const T E4 = fma(F3, r4, F2 * (r0));
  const T E5 = F3 * (r5);
  const T E6 = F3 * (r6);
  const T E7 = fma(F3, r7, F2 * (r0));
  const T E8 = F3 * (r8);
  const T E9 = fma(F3, r9, F2 * (r0));
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  nu[0] = fma(rl, E0, nu[0]);
  nu[1] = fma(lx, E0, fma(rl, E1, nu[1]));
  nu[2] = fma(ly, E0, fma(rl, E2, nu[2]));
  nu[3] = fma(lz, E0, fma(rl, E3, nu[3]));
  nu[4] = fma((lx * T(2)), E1, fma(rl, E4, nu[4]));
  nu[5] = fma(ly, E1, fma(lx, E2, fma(rl, E5, nu[5])));
  nu[6] = fma(lz, E1, fma(lx, E3, fma(rl, E6, nu[6])));
  nu[7] = fma((ly * T(2)), E2, fma(rl, E7, nu[7]));
  nu[8] = fma(lz, E2, fma(ly, E3, fma(rl, E8, nu[8])));
  nu[9] = fma((lz * T(2)), E3, fma(rl, E9, nu[9]));
}

__device__ __forceinline__ void m2m_adj_acc_p2(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {
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
  nuc[0] = fma(w9, nup[9], fma(w8, nup[8], fma(w7, nup[7], fma(w6, nup[6], fma(w5, nup[5], fma(w4, nup[4], fma(w3, nup[3], fma(w2, nup[2], fma(w1, nup[1], fma(w0, nup[0], nuc[0]))))))))));
  nuc[1] = fma(w3, nup[6], fma(w2, nup[5], fma(w1 * 2.0, nup[4], fma(w0, nup[1], nuc[1]))));
  nuc[2] = fma(w3, nup[8], fma(w2 * 2.0, nup[7], fma(w1, nup[5], fma(w0, nup[2], nuc[2]))));
  nuc[3] = fma(w3 * 2.0, nup[9], fma(w2, nup[8], fma(w1, nup[6], fma(w0, nup[3], nuc[3]))));
  nuc[4] = fma(w0, nup[4], nuc[4]);
  nuc[5] = fma(w0, nup[5], nuc[5]);
  nuc[6] = fma(w0, nup[6], nuc[6]);
  nuc[7] = fma(w0, nup[7], nuc[7]);
  nuc[8] = fma(w0, nup[8], nuc[8]);
  nuc[9] = fma(w0, nup[9], nuc[9]);
}

__device__ __forceinline__ void p2m_adj_p2(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {
  const double q0 = 1.0;
  const double q1 = q0 * dx;
  const double q2 = q0 * dy;
  const double q3 = q0 * dz;
  gx = fma(m, fma(nu[6], q3, fma(nu[5], q2, fma(nu[4] * 2.0, q1, fma(nu[1], q0, 0.0)))), gx);
  gy = fma(m, fma(nu[8], q3, fma(nu[7] * 2.0, q2, fma(nu[5], q1, fma(nu[2], q0, 0.0)))), gy);
  gz = fma(m, fma(nu[9] * 2.0, q3, fma(nu[8], q2, fma(nu[6], q1, fma(nu[3], q0, 0.0)))), gz);
}

template <typename T>
__device__ __forceinline__ void m2p_adj_self_p3(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T F5 = F4 * (T(-9) * is);
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
  T q1 = lx;
  T q2 = ly;
  T q3 = lz;
  T q4 = lx * m1;
  T q5 = lx * m2;
  q5 = fma(ly, m1, q5);
  T q6 = lx * m3;
  q6 = fma(lz, m1, q6);
  T q7 = ly * m2;
  T q8 = ly * m3;
  q8 = fma(lz, m2, q8);
  T q9 = lz * m3;
  T S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, H2x, H2y, H2z, S3, G3x, H3x, G3y, H3y, G3z, H3z;
  { const T b = B[0];
    S0 = b;
  }
  { const T b = B[1];
    S1 = b;
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = b;
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = b;
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = b;
  }
  { const T b = B[5];
    S2 = b * m1;
    G2x = b;
  }
  { const T b = B[6];
    S2 = fma(b, m2, S2);
    G2y = b;
  }
  { const T b = B[7];
    S2 = fma(b, m3, S2);
    G2z = b;
  }
  { const T b = B[8];
    S2 = fma(b, m4, S2);
    G2x = fma(b, m1, G2x);
    H2x = b * q1;
  }
  { const T b = B[9];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    H2x = fma(b, q2, H2x);
    G2y = fma(b, m1, G2y);
    H2y = b * q1;
  }
  { const T b = B[10];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    H2x = fma(b, q3, H2x);
    G2z = fma(b, m1, G2z);
    H2z = b * q1;
  }
  { const T b = B[11];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
    H2y = fma(b, q2, H2y);
  }
  { const T b = B[12];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    H2y = fma(b, q3, H2y);
    G2z = fma(b, m2, G2z);
    H2z = fma(b, q2, H2z);
  }
  { const T b = B[13];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
    H2z = fma(b, q3, H2z);
  }
  { const T b = B[14];
    S3 = b * m10;
    G3x = b * m4;
    H3x = b * q4;
  }
  { const T b = B[15];
    S3 = fma(b, m11, S3);
    G3x = fma(b, m5, G3x);
    H3x = fma(b, q5, H3x);
    G3y = b * m4;
    H3y = b * q4;
  }
  { const T b = B[16];
    S3 = fma(b, m12, S3);
    G3x = fma(b, m6, G3x);
    H3x = fma(b, q6, H3x);
    G3z = b * m4;
    H3z = b * q4;
  }
  { const T b = B[17];
    S3 = fma(b, m13, S3);
    G3x = fma(b, m7, G3x);
    H3x = fma(b, q7, H3x);
    G3y = fma(b, m5, G3y);
    H3y = fma(b, q5, H3y);
  }
  { const T b = B[18];
    S3 = fma(b, m14, S3);
    G3x = fma(b, m8, G3x);
    H3x = fma(b, q8, H3x);
    G3y = fma(b, m6, G3y);
    H3y = fma(b, q6, H3y);
    G3z = fma(b, m5, G3z);
    H3z = fma(b, q5, H3z);
  }
  { const T b = B[19];
    S3 = fma(b, m15, S3);
    G3x = fma(b, m9, G3x);
    H3x = fma(b, q9, H3x);
    G3z = fma(b, m6, G3z);
    H3z = fma(b, q6, H3z);
  }
  { const T b = B[20];
    S3 = fma(b, m16, S3);
    G3y = fma(b, m7, G3y);
    H3y = fma(b, q7, H3y);
  }
  { const T b = B[21];
    S3 = fma(b, m17, S3);
    G3y = fma(b, m8, G3y);
    H3y = fma(b, q8, H3y);
    G3z = fma(b, m7, G3z);
    H3z = fma(b, q7, H3z);
  }
  { const T b = B[22];
    S3 = fma(b, m18, S3);
    G3y = fma(b, m9, G3y);
    H3y = fma(b, q9, H3y);
    G3z = fma(b, m8, G3z);
    H3z = fma(b, q8, H3z);
  }
  { const T b = B[23];
    S3 = fma(b, m19, S3);
    G3z = fma(b, m9, G3z);
    H3z = fma(b, q9, H3z);
  }
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  T ax = ox, ay = oy, az = oz;
  { const T a1 = F1 * S0;  // F_{j+1} S_j
    const T c1 = F2 * S0 * rl;  // R_k coefficient
    ax = fma(a1, lx, fma(Rx, c1, ax));
    ay = fma(a1, ly, fma(Ry, c1, ay));
    az = fma(a1, lz, fma(Rz, c1, az));
  }
  { const T a1 = F2 * S1;  // F_{j+1} S_j
    const T gl = fma(G1x, lx, fma(G1y, ly, G1z * lz));
    const T c1 = fma(F3 * S1, rl, F2 * gl);  // R_k coefficient
    const T c2 = F2 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G1x, ax)));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G1y, ay)));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G1z, az)));
  }
  { const T a1 = F3 * S2;  // F_{j+1} S_j
    const T gl = fma(G2x, lx, fma(G2y, ly, G2z * lz));
    const T c1 = fma(F4 * S2, rl, F3 * gl);  // R_k coefficient
    const T c2 = F3 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G2x, fma(F2, H2x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G2y, fma(F2, H2y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G2z, fma(F2, H2z, az))));
  }
  { const T a1 = F4 * S3;  // F_{j+1} S_j
    const T gl = fma(G3x, lx, fma(G3y, ly, G3z * lz));
    const T c1 = fma(F5 * S3, rl, F4 * gl);  // R_k coefficient
    const T c2 = F4 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G3x, fma(F3, H3x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G3y, fma(F3, H3y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G3z, fma(F3, H3z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

__device__ __forceinline__ void m2p2_adj_self_p3(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz, float2 eps2, float2 lx, float2 ly, float2 lz, float2& ox, float2& oy, float2& oz) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = nbody_rsqrt2(s);
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 F4 = __fmul2_rn(F3, __fmul2_rn(make_float2(-7.0f, -7.0f), is));
  const float2 F5 = __fmul2_rn(F4, __fmul2_rn(make_float2(-9.0f, -9.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Rx_3 = __fmul2_rn(Rx, make_float2(0.333333333f, 0.333333333f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Ry_3 = __fmul2_rn(Ry, make_float2(0.333333333f, 0.333333333f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 Rz_3 = __fmul2_rn(Rz, make_float2(0.333333333f, 0.333333333f));
  const float2 m0 = make_float2(1.0f, 1.0f);
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
  float2 q1 = lx;
  float2 q2 = ly;
  float2 q3 = lz;
  float2 q4 = __fmul2_rn(lx, m1);
  float2 q5 = __fmul2_rn(lx, m2);
  q5 = __ffma2_rn(ly, m1, q5);
  float2 q6 = __fmul2_rn(lx, m3);
  q6 = __ffma2_rn(lz, m1, q6);
  float2 q7 = __fmul2_rn(ly, m2);
  float2 q8 = __fmul2_rn(ly, m3);
  q8 = __ffma2_rn(lz, m2, q8);
  float2 q9 = __fmul2_rn(lz, m3);
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, H2x, H2y, H2z, S3, G3x, H3x, G3y, H3y, G3z, H3z;
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
    H2x = __fmul2_rn(b, q1);
  }
  { const float2 b = B[9];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    H2x = __ffma2_rn(b, q2, H2x);
    G2y = __ffma2_rn(b, m1, G2y);
    H2y = __fmul2_rn(b, q1);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    H2x = __ffma2_rn(b, q3, H2x);
    G2z = __ffma2_rn(b, m1, G2z);
    H2z = __fmul2_rn(b, q1);
  }
  { const float2 b = B[11];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
    H2y = __ffma2_rn(b, q2, H2y);
  }
  { const float2 b = B[12];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    H2y = __ffma2_rn(b, q3, H2y);
    G2z = __ffma2_rn(b, m2, G2z);
    H2z = __ffma2_rn(b, q2, H2z);
  }
  { const float2 b = B[13];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
    H2z = __ffma2_rn(b, q3, H2z);
  }
  { const float2 b = B[14];
    S3 = __fmul2_rn(b, m10);
    G3x = __fmul2_rn(b, m4);
    H3x = __fmul2_rn(b, q4);
  }
  { const float2 b = B[15];
    S3 = __ffma2_rn(b, m11, S3);
    G3x = __ffma2_rn(b, m5, G3x);
    H3x = __ffma2_rn(b, q5, H3x);
    G3y = __fmul2_rn(b, m4);
    H3y = __fmul2_rn(b, q4);
  }
  { const float2 b = B[16];
    S3 = __ffma2_rn(b, m12, S3);
    G3x = __ffma2_rn(b, m6, G3x);
    H3x = __ffma2_rn(b, q6, H3x);
    G3z = __fmul2_rn(b, m4);
    H3z = __fmul2_rn(b, q4);
  }
  { const float2 b = B[17];
    S3 = __ffma2_rn(b, m13, S3);
    G3x = __ffma2_rn(b, m7, G3x);
    H3x = __ffma2_rn(b, q7, H3x);
    G3y = __ffma2_rn(b, m5, G3y);
    H3y = __ffma2_rn(b, q5, H3y);
  }
  { const float2 b = B[18];
    S3 = __ffma2_rn(b, m14, S3);
    G3x = __ffma2_rn(b, m8, G3x);
    H3x = __ffma2_rn(b, q8, H3x);
    G3y = __ffma2_rn(b, m6, G3y);
    H3y = __ffma2_rn(b, q6, H3y);
    G3z = __ffma2_rn(b, m5, G3z);
    H3z = __ffma2_rn(b, q5, H3z);
  }
  { const float2 b = B[19];
    S3 = __ffma2_rn(b, m15, S3);
    G3x = __ffma2_rn(b, m9, G3x);
    H3x = __ffma2_rn(b, q9, H3x);
    G3z = __ffma2_rn(b, m6, G3z);
    H3z = __ffma2_rn(b, q6, H3z);
  }
  { const float2 b = B[20];
    S3 = __ffma2_rn(b, m16, S3);
    G3y = __ffma2_rn(b, m7, G3y);
    H3y = __ffma2_rn(b, q7, H3y);
  }
  { const float2 b = B[21];
    S3 = __ffma2_rn(b, m17, S3);
    G3y = __ffma2_rn(b, m8, G3y);
    H3y = __ffma2_rn(b, q8, H3y);
    G3z = __ffma2_rn(b, m7, G3z);
    H3z = __ffma2_rn(b, q7, H3z);
  }
  { const float2 b = B[22];
    S3 = __ffma2_rn(b, m18, S3);
    G3y = __ffma2_rn(b, m9, G3y);
    H3y = __ffma2_rn(b, q9, H3y);
    G3z = __ffma2_rn(b, m8, G3z);
    H3z = __ffma2_rn(b, q8, H3z);
  }
  { const float2 b = B[23];
    S3 = __ffma2_rn(b, m19, S3);
    G3z = __ffma2_rn(b, m9, G3z);
    H3z = __ffma2_rn(b, q9, H3z);
  }
  const float2 rl = __ffma2_rn(Rx, lx, __ffma2_rn(Ry, ly, __fmul2_rn(Rz, lz)));
  float2 ax = ox, ay = oy, az = oz;
  { const float2 a1 = __fmul2_rn(F1, S0);
    const float2 c1 = __fmul2_rn(__fmul2_rn(F2, S0), rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, ax));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, ay));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, az));
  }
  { const float2 a1 = __fmul2_rn(F2, S1);
    const float2 gl = __ffma2_rn(G1x, lx, __ffma2_rn(G1y, ly, __fmul2_rn(G1z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F3, S1), rl, __fmul2_rn(F2, gl));
    const float2 c2 = __fmul2_rn(F2, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G1x, ax)));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G1y, ay)));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G1z, az)));
  }
  { const float2 a1 = __fmul2_rn(F3, S2);
    const float2 gl = __ffma2_rn(G2x, lx, __ffma2_rn(G2y, ly, __fmul2_rn(G2z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F4, S2), rl, __fmul2_rn(F3, gl));
    const float2 c2 = __fmul2_rn(F3, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G2x, __ffma2_rn(F2, H2x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G2y, __ffma2_rn(F2, H2y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G2z, __ffma2_rn(F2, H2z, az))));
  }
  { const float2 a1 = __fmul2_rn(F4, S3);
    const float2 gl = __ffma2_rn(G3x, lx, __ffma2_rn(G3y, ly, __fmul2_rn(G3z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F5, S3), rl, __fmul2_rn(F4, gl));
    const float2 c2 = __fmul2_rn(F4, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G3x, __ffma2_rn(F3, H3x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G3y, __ffma2_rn(F3, H3y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G3z, __ffma2_rn(F3, H3z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

template <typename T>
__device__ __forceinline__ void m2p_adj_src_p3(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz,
                                         T* __restrict__ nu) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T r0 = T(1);
  const T r1 = Rx;
  const T r2 = Ry;
  const T r3 = Rz;
  const T r4 = r1 * Rx;
  const T r5 = r2 * Rx;
  const T r6 = r3 * Rx;
  const T r7 = r2 * Ry;
  const T r8 = r3 * Ry;
  const T r9 = r3 * Rz;
  const T r10 = r4 * Rx;
  const T r11 = r5 * Rx;
  const T r12 = r6 * Rx;
  const T r13 = r7 * Rx;
  const T r14 = r8 * Rx;
  const T r15 = r9 * Rx;
  const T r16 = r7 * Ry;
  const T r17 = r8 * Ry;
  const T r18 = r9 * Ry;
  const T r19 = r9 * Rz;
  const T E0 = F1 * (r0);
  const T E1 = F2 * (r1);
  const T E2 = F2 * (r2);
  const T E3 = F2 * (r3);
  const T E4 = fma(F3, r4, F2 * (r0));
  const T E5 = F3 * (r5);
  const T E6 = F3 * (r6);
  const T E7 = fma(F3, r7, F2 * (r0));
  const T E8 = F3 * (r8);
  const T E9 = fma(F3, r9, F2 * (r0));
  const T E10 = fma(F4, r10, F3 * (r1 * T(3)));
  const T E11 = fma(F4, r11, F3 * (r2));
  const T E12 = fma(F4, r12, F3 * (r3));
  const T E13 = fma(F4, r13, F3 * (r1));
  const T E14 = F4 * (r14);
  const T E15 = fma(F4, r15, F3 * (r1));
  const T E16 = fma(F4, r16, F3 * (r2 * T(3)));
  const T E17 = fma(F4, r17, F3 * (r3));
  const T E18 = fma(F4, r18, F3 * (r2));
  const T E19 = fma(F4, r19, F3 * (r3 * T(3)));
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  nu[0] = fma(rl, E0, nu[0]);
  nu[1] = fma(lx, E0, fma(rl, E1, nu[1]));
  nu[2] = fma(ly, E0, fma(rl, E2, nu[2]));
  nu[3] = fma(lz, E0, fma(rl, E3, nu[3]));
  nu[4] = fma((lx * T(2)), E1, fma(rl, E4, nu[4]));
  nu[5] = fma(ly, E1, fma(lx, E2, fma(rl, E5, nu[5])));
  nu[6] = fma(lz, E1, fma(lx, E3, fma(rl, E6, nu[6])));
  nu[7] = fma((ly * T(2)), E2, fma(rl, E7, nu[7]));
  nu[8] = fma(lz, E2, fma(ly, E3, fma(rl, E8, nu[8])));
  nu[9] = fma((lz * T(2)), E3, fma(rl, E9, nu[9]));
  nu[10] = fma((lx * T(3)), E4, fma(rl, E10, nu[10]));
  nu[11] = fma(ly, E4, fma((lx * T(2)), E5, fma(rl, E11, nu[11])));
  nu[12] = fma(lz, E4, fma((lx * T(2)), E6, fma(rl, E12, nu[12])));
  nu[13] = fma((ly * T(2)), E5, fma(lx, E7, fma(rl, E13, nu[13])));
  nu[14] = fma(lz, E5, fma(ly, E6, fma(lx, E8, fma(rl, E14, nu[14]))));
  nu[15] = fma((lz * T(2)), E6, fma(lx, E9, fma(rl, E15, nu[15])));
  nu[16] = fma((ly * T(3)), E7, fma(rl, E16, nu[16]));
  nu[17] = fma(lz, E7, fma((ly * T(2)), E8, fma(rl, E17, nu[17])));
  nu[18] = fma((lz * T(2)), E8, fma(ly, E9, fma(rl, E18, nu[18])));
  nu[19] = fma((lz * T(3)), E9, fma(rl, E19, nu[19]));
}

__device__ __forceinline__ void m2m_adj_acc_p3(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {
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
  nuc[0] = fma(w19, nup[19], fma(w18, nup[18], fma(w17, nup[17], fma(w16, nup[16], fma(w15, nup[15], fma(w14, nup[14], fma(w13, nup[13], fma(w12, nup[12], fma(w11, nup[11], fma(w10, nup[10], fma(w9, nup[9], fma(w8, nup[8], fma(w7, nup[7], fma(w6, nup[6], fma(w5, nup[5], fma(w4, nup[4], fma(w3, nup[3], fma(w2, nup[2], fma(w1, nup[1], fma(w0, nup[0], nuc[0]))))))))))))))))))));
  nuc[1] = fma(w9, nup[15], fma(w8, nup[14], fma(w7, nup[13], fma(w6 * 2.0, nup[12], fma(w5 * 2.0, nup[11], fma(w4 * 3.0, nup[10], fma(w3, nup[6], fma(w2, nup[5], fma(w1 * 2.0, nup[4], fma(w0, nup[1], nuc[1]))))))))));
  nuc[2] = fma(w9, nup[18], fma(w8 * 2.0, nup[17], fma(w7 * 3.0, nup[16], fma(w6, nup[14], fma(w5 * 2.0, nup[13], fma(w4, nup[11], fma(w3, nup[8], fma(w2 * 2.0, nup[7], fma(w1, nup[5], fma(w0, nup[2], nuc[2]))))))))));
  nuc[3] = fma(w9 * 3.0, nup[19], fma(w8 * 2.0, nup[18], fma(w7, nup[17], fma(w6 * 2.0, nup[15], fma(w5, nup[14], fma(w4, nup[12], fma(w3 * 2.0, nup[9], fma(w2, nup[8], fma(w1, nup[6], fma(w0, nup[3], nuc[3]))))))))));
  nuc[4] = fma(w3, nup[12], fma(w2, nup[11], fma(w1 * 3.0, nup[10], fma(w0, nup[4], nuc[4]))));
  nuc[5] = fma(w3, nup[14], fma(w2 * 2.0, nup[13], fma(w1 * 2.0, nup[11], fma(w0, nup[5], nuc[5]))));
  nuc[6] = fma(w3 * 2.0, nup[15], fma(w2, nup[14], fma(w1 * 2.0, nup[12], fma(w0, nup[6], nuc[6]))));
  nuc[7] = fma(w3, nup[17], fma(w2 * 3.0, nup[16], fma(w1, nup[13], fma(w0, nup[7], nuc[7]))));
  nuc[8] = fma(w3 * 2.0, nup[18], fma(w2 * 2.0, nup[17], fma(w1, nup[14], fma(w0, nup[8], nuc[8]))));
  nuc[9] = fma(w3 * 3.0, nup[19], fma(w2, nup[18], fma(w1, nup[15], fma(w0, nup[9], nuc[9]))));
  nuc[10] = fma(w0, nup[10], nuc[10]);
  nuc[11] = fma(w0, nup[11], nuc[11]);
  nuc[12] = fma(w0, nup[12], nuc[12]);
  nuc[13] = fma(w0, nup[13], nuc[13]);
  nuc[14] = fma(w0, nup[14], nuc[14]);
  nuc[15] = fma(w0, nup[15], nuc[15]);
  nuc[16] = fma(w0, nup[16], nuc[16]);
  nuc[17] = fma(w0, nup[17], nuc[17]);
  nuc[18] = fma(w0, nup[18], nuc[18]);
  nuc[19] = fma(w0, nup[19], nuc[19]);
}

__device__ __forceinline__ void p2m_adj_p3(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {
  const double q0 = 1.0;
  const double q1 = q0 * dx;
  const double q2 = q0 * dy;
  const double q3 = q0 * dz;
  const double q4 = q1 * dx;
  const double q5 = q2 * dx;
  const double q6 = q3 * dx;
  const double q7 = q2 * dy;
  const double q8 = q3 * dy;
  const double q9 = q3 * dz;
  gx = fma(m, fma(nu[15], q9, fma(nu[14], q8, fma(nu[13], q7, fma(nu[12] * 2.0, q6, fma(nu[11] * 2.0, q5, fma(nu[10] * 3.0, q4, fma(nu[6], q3, fma(nu[5], q2, fma(nu[4] * 2.0, q1, fma(nu[1], q0, 0.0)))))))))), gx);
  gy = fma(m, fma(nu[18], q9, fma(nu[17] * 2.0, q8, fma(nu[16] * 3.0, q7, fma(nu[14], q6, fma(nu[13] * 2.0, q5, fma(nu[11], q4, fma(nu[8], q3, fma(nu[7] * 2.0, q2, fma(nu[5], q1, fma(nu[2], q0, 0.0)))))))))), gy);
  gz = fma(m, fma(nu[19] * 3.0, q9, fma(nu[18] * 2.0, q8, fma(nu[17], q7, fma(nu[15] * 2.0, q6, fma(nu[14], q5, fma(nu[12], q4, fma(nu[9] * 2.0, q3, fma(nu[8], q2, fma(nu[6], q1, fma(nu[3], q0, 0.0)))))))))), gz);
}

template <typename T>
__device__ __forceinline__ void m2p_adj_self_p4(const T* __restrict__ B, T Rx, T Ry, T Rz, T eps2,
                                          T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T F5 = F4 * (T(-9) * is);
  const T F6 = F5 * (T(-11) * is);
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
  T q1 = lx;
  T q2 = ly;
  T q3 = lz;
  T q4 = lx * m1;
  T q5 = lx * m2;
  q5 = fma(ly, m1, q5);
  T q6 = lx * m3;
  q6 = fma(lz, m1, q6);
  T q7 = ly * m2;
  T q8 = ly * m3;
  q8 = fma(lz, m2, q8);
  T q9 = lz * m3;
  T q10 = lx * m4;
  T q11 = lx * m5;
  q11 = fma(ly, m4, q11);
  T q12 = lx * m6;
  q12 = fma(lz, m4, q12);
  T q13 = lx * m7;
  q13 = fma(ly, m5, q13);
  T q14 = lx * m8;
  q14 = fma(ly, m6, q14);
  q14 = fma(lz, m5, q14);
  T q15 = lx * m9;
  q15 = fma(lz, m6, q15);
  T q16 = ly * m7;
  T q17 = ly * m8;
  q17 = fma(lz, m7, q17);
  T q18 = ly * m9;
  q18 = fma(lz, m8, q18);
  T q19 = lz * m9;
  T S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, H2x, H2y, H2z, S3, G3x, H3x, G3y, H3y, G3z, H3z, S4, G4x, H4x, G4y, H4y, G4z, H4z;
  { const T b = B[0];
    S0 = b;
  }
  { const T b = B[1];
    S1 = b;
  }
  { const T b = B[2];
    S1 = fma(b, m1, S1);
    G1x = b;
  }
  { const T b = B[3];
    S1 = fma(b, m2, S1);
    G1y = b;
  }
  { const T b = B[4];
    S1 = fma(b, m3, S1);
    G1z = b;
  }
  { const T b = B[5];
    S2 = b;
  }
  { const T b = B[6];
    S2 = fma(b, m1, S2);
    G2x = b;
  }
  { const T b = B[7];
    S2 = fma(b, m2, S2);
    G2y = b;
  }
  { const T b = B[8];
    S2 = fma(b, m3, S2);
    G2z = b;
  }
  { const T b = B[9];
    S2 = fma(b, m4, S2);
    G2x = fma(b, m1, G2x);
    H2x = b * q1;
  }
  { const T b = B[10];
    S2 = fma(b, m5, S2);
    G2x = fma(b, m2, G2x);
    H2x = fma(b, q2, H2x);
    G2y = fma(b, m1, G2y);
    H2y = b * q1;
  }
  { const T b = B[11];
    S2 = fma(b, m6, S2);
    G2x = fma(b, m3, G2x);
    H2x = fma(b, q3, H2x);
    G2z = fma(b, m1, G2z);
    H2z = b * q1;
  }
  { const T b = B[12];
    S2 = fma(b, m7, S2);
    G2y = fma(b, m2, G2y);
    H2y = fma(b, q2, H2y);
  }
  { const T b = B[13];
    S2 = fma(b, m8, S2);
    G2y = fma(b, m3, G2y);
    H2y = fma(b, q3, H2y);
    G2z = fma(b, m2, G2z);
    H2z = fma(b, q2, H2z);
  }
  { const T b = B[14];
    S2 = fma(b, m9, S2);
    G2z = fma(b, m3, G2z);
    H2z = fma(b, q3, H2z);
  }
  { const T b = B[15];
    S3 = b * m4;
    G3x = b * m1;
    H3x = b * q1;
  }
  { const T b = B[16];
    S3 = fma(b, m5, S3);
    G3x = fma(b, m2, G3x);
    H3x = fma(b, q2, H3x);
    G3y = b * m1;
    H3y = b * q1;
  }
  { const T b = B[17];
    S3 = fma(b, m6, S3);
    G3x = fma(b, m3, G3x);
    H3x = fma(b, q3, H3x);
    G3z = b * m1;
    H3z = b * q1;
  }
  { const T b = B[18];
    S3 = fma(b, m7, S3);
    G3y = fma(b, m2, G3y);
    H3y = fma(b, q2, H3y);
  }
  { const T b = B[19];
    S3 = fma(b, m8, S3);
    G3y = fma(b, m3, G3y);
    H3y = fma(b, q3, H3y);
    G3z = fma(b, m2, G3z);
    H3z = fma(b, q2, H3z);
  }
  { const T b = B[20];
    S3 = fma(b, m9, S3);
    G3z = fma(b, m3, G3z);
    H3z = fma(b, q3, H3z);
  }
  { const T b = B[21];
    S3 = fma(b, m10, S3);
    G3x = fma(b, m4, G3x);
    H3x = fma(b, q4, H3x);
  }
  { const T b = B[22];
    S3 = fma(b, m11, S3);
    G3x = fma(b, m5, G3x);
    H3x = fma(b, q5, H3x);
    G3y = fma(b, m4, G3y);
    H3y = fma(b, q4, H3y);
  }
  { const T b = B[23];
    S3 = fma(b, m12, S3);
    G3x = fma(b, m6, G3x);
    H3x = fma(b, q6, H3x);
    G3z = fma(b, m4, G3z);
    H3z = fma(b, q4, H3z);
  }
  { const T b = B[24];
    S3 = fma(b, m13, S3);
    G3x = fma(b, m7, G3x);
    H3x = fma(b, q7, H3x);
    G3y = fma(b, m5, G3y);
    H3y = fma(b, q5, H3y);
  }
  { const T b = B[25];
    S3 = fma(b, m14, S3);
    G3x = fma(b, m8, G3x);
    H3x = fma(b, q8, H3x);
    G3y = fma(b, m6, G3y);
    H3y = fma(b, q6, H3y);
    G3z = fma(b, m5, G3z);
    H3z = fma(b, q5, H3z);
  }
  { const T b = B[26];
    S3 = fma(b, m15, S3);
    G3x = fma(b, m9, G3x);
    H3x = fma(b, q9, H3x);
    G3z = fma(b, m6, G3z);
    H3z = fma(b, q6, H3z);
  }
  { const T b = B[27];
    S3 = fma(b, m16, S3);
    G3y = fma(b, m7, G3y);
    H3y = fma(b, q7, H3y);
  }
  { const T b = B[28];
    S3 = fma(b, m17, S3);
    G3y = fma(b, m8, G3y);
    H3y = fma(b, q8, H3y);
    G3z = fma(b, m7, G3z);
    H3z = fma(b, q7, H3z);
  }
  { const T b = B[29];
    S3 = fma(b, m18, S3);
    G3y = fma(b, m9, G3y);
    H3y = fma(b, q9, H3y);
    G3z = fma(b, m8, G3z);
    H3z = fma(b, q8, H3z);
  }
  { const T b = B[30];
    S3 = fma(b, m19, S3);
    G3z = fma(b, m9, G3z);
    H3z = fma(b, q9, H3z);
  }
  { const T b = B[31];
    S4 = b * m20;
    G4x = b * m10;
    H4x = b * q10;
  }
  { const T b = B[32];
    S4 = fma(b, m21, S4);
    G4x = fma(b, m11, G4x);
    H4x = fma(b, q11, H4x);
    G4y = b * m10;
    H4y = b * q10;
  }
  { const T b = B[33];
    S4 = fma(b, m22, S4);
    G4x = fma(b, m12, G4x);
    H4x = fma(b, q12, H4x);
    G4z = b * m10;
    H4z = b * q10;
  }
  { const T b = B[34];
    S4 = fma(b, m23, S4);
    G4x = fma(b, m13, G4x);
    H4x = fma(b, q13, H4x);
    G4y = fma(b, m11, G4y);
    H4y = fma(b, q11, H4y);
  }
  { const T b = B[35];
    S4 = fma(b, m24, S4);
    G4x = fma(b, m14, G4x);
    H4x = fma(b, q14, H4x);
    G4y = fma(b, m12, G4y);
    H4y = fma(b, q12, H4y);
    G4z = fma(b, m11, G4z);
    H4z = fma(b, q11, H4z);
  }
  { const T b = B[36];
    S4 = fma(b, m25, S4);
    G4x = fma(b, m15, G4x);
    H4x = fma(b, q15, H4x);
    G4z = fma(b, m12, G4z);
    H4z = fma(b, q12, H4z);
  }
  { const T b = B[37];
    S4 = fma(b, m26, S4);
    G4x = fma(b, m16, G4x);
    H4x = fma(b, q16, H4x);
    G4y = fma(b, m13, G4y);
    H4y = fma(b, q13, H4y);
  }
  { const T b = B[38];
    S4 = fma(b, m27, S4);
    G4x = fma(b, m17, G4x);
    H4x = fma(b, q17, H4x);
    G4y = fma(b, m14, G4y);
    H4y = fma(b, q14, H4y);
    G4z = fma(b, m13, G4z);
    H4z = fma(b, q13, H4z);
  }
  { const T b = B[39];
    S4 = fma(b, m28, S4);
    G4x = fma(b, m18, G4x);
    H4x = fma(b, q18, H4x);
    G4y = fma(b, m15, G4y);
    H4y = fma(b, q15, H4y);
    G4z = fma(b, m14, G4z);
    H4z = fma(b, q14, H4z);
  }
  { const T b = B[40];
    S4 = fma(b, m29, S4);
    G4x = fma(b, m19, G4x);
    H4x = fma(b, q19, H4x);
    G4z = fma(b, m15, G4z);
    H4z = fma(b, q15, H4z);
  }
  { const T b = B[41];
    S4 = fma(b, m30, S4);
    G4y = fma(b, m16, G4y);
    H4y = fma(b, q16, H4y);
  }
  { const T b = B[42];
    S4 = fma(b, m31, S4);
    G4y = fma(b, m17, G4y);
    H4y = fma(b, q17, H4y);
    G4z = fma(b, m16, G4z);
    H4z = fma(b, q16, H4z);
  }
  { const T b = B[43];
    S4 = fma(b, m32, S4);
    G4y = fma(b, m18, G4y);
    H4y = fma(b, q18, H4y);
    G4z = fma(b, m17, G4z);
    H4z = fma(b, q17, H4z);
  }
  { const T b = B[44];
    S4 = fma(b, m33, S4);
    G4y = fma(b, m19, G4y);
    H4y = fma(b, q19, H4y);
    G4z = fma(b, m18, G4z);
    H4z = fma(b, q18, H4z);
  }
  { const T b = B[45];
    S4 = fma(b, m34, S4);
    G4z = fma(b, m19, G4z);
    H4z = fma(b, q19, H4z);
  }
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  T ax = ox, ay = oy, az = oz;
  { const T a1 = F1 * S0;  // F_{j+1} S_j
    const T c1 = F2 * S0 * rl;  // R_k coefficient
    ax = fma(a1, lx, fma(Rx, c1, ax));
    ay = fma(a1, ly, fma(Ry, c1, ay));
    az = fma(a1, lz, fma(Rz, c1, az));
  }
  { const T a1 = F2 * S1;  // F_{j+1} S_j
    const T gl = fma(G1x, lx, fma(G1y, ly, G1z * lz));
    const T c1 = fma(F3 * S1, rl, F2 * gl);  // R_k coefficient
    const T c2 = F2 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G1x, ax)));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G1y, ay)));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G1z, az)));
  }
  { const T a1 = F3 * S2;  // F_{j+1} S_j
    const T gl = fma(G2x, lx, fma(G2y, ly, G2z * lz));
    const T c1 = fma(F4 * S2, rl, F3 * gl);  // R_k coefficient
    const T c2 = F3 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G2x, fma(F2, H2x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G2y, fma(F2, H2y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G2z, fma(F2, H2z, az))));
  }
  { const T a1 = F4 * S3;  // F_{j+1} S_j
    const T gl = fma(G3x, lx, fma(G3y, ly, G3z * lz));
    const T c1 = fma(F5 * S3, rl, F4 * gl);  // R_k coefficient
    const T c2 = F4 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G3x, fma(F3, H3x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G3y, fma(F3, H3y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G3z, fma(F3, H3z, az))));
  }
  { const T a1 = F5 * S4;  // F_{j+1} S_j
    const T gl = fma(G4x, lx, fma(G4y, ly, G4z * lz));
    const T c1 = fma(F6 * S4, rl, F5 * gl);  // R_k coefficient
    const T c2 = F5 * rl;  // G_{j,k} coefficient
    ax = fma(a1, lx, fma(Rx, c1, fma(c2, G4x, fma(F4, H4x, ax))));
    ay = fma(a1, ly, fma(Ry, c1, fma(c2, G4y, fma(F4, H4y, ay))));
    az = fma(a1, lz, fma(Rz, c1, fma(c2, G4z, fma(F4, H4z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

__device__ __forceinline__ void m2p2_adj_self_p4(const float2* __restrict__ B, float2 Rx, float2 Ry, float2 Rz, float2 eps2, float2 lx, float2 ly, float2 lz, float2& ox, float2& oy, float2& oz) {
  const float2 s = __ffma2_rn(Rx, Rx, __ffma2_rn(Ry, Ry, __ffma2_rn(Rz, Rz, eps2)));
  const float2 F0 = nbody_rsqrt2(s);
  const float2 is = __fmul2_rn(F0, F0);
  const float2 F1 = __fmul2_rn(F0, __fmul2_rn(make_float2(-1.0f, -1.0f), is));
  const float2 F2 = __fmul2_rn(F1, __fmul2_rn(make_float2(-3.0f, -3.0f), is));
  const float2 F3 = __fmul2_rn(F2, __fmul2_rn(make_float2(-5.0f, -5.0f), is));
  const float2 F4 = __fmul2_rn(F3, __fmul2_rn(make_float2(-7.0f, -7.0f), is));
  const float2 F5 = __fmul2_rn(F4, __fmul2_rn(make_float2(-9.0f, -9.0f), is));
  const float2 F6 = __fmul2_rn(F5, __fmul2_rn(make_float2(-11.0f, -11.0f), is));
  const float2 Rx_2 = __fmul2_rn(Rx, make_float2(0.5f, 0.5f));
  const float2 Rx_3 = __fmul2_rn(Rx, make_float2(0.333333333f, 0.333333333f));
  const float2 Rx_4 = __fmul2_rn(Rx, make_float2(0.25f, 0.25f));
  const float2 Ry_2 = __fmul2_rn(Ry, make_float2(0.5f, 0.5f));
  const float2 Ry_3 = __fmul2_rn(Ry, make_float2(0.333333333f, 0.333333333f));
  const float2 Ry_4 = __fmul2_rn(Ry, make_float2(0.25f, 0.25f));
  const float2 Rz_2 = __fmul2_rn(Rz, make_float2(0.5f, 0.5f));
  const float2 Rz_3 = __fmul2_rn(Rz, make_float2(0.333333333f, 0.333333333f));
  const float2 Rz_4 = __fmul2_rn(Rz, make_float2(0.25f, 0.25f));
  const float2 m0 = make_float2(1.0f, 1.0f);
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
  float2 q1 = lx;
  float2 q2 = ly;
  float2 q3 = lz;
  float2 q4 = __fmul2_rn(lx, m1);
  float2 q5 = __fmul2_rn(lx, m2);
  q5 = __ffma2_rn(ly, m1, q5);
  float2 q6 = __fmul2_rn(lx, m3);
  q6 = __ffma2_rn(lz, m1, q6);
  float2 q7 = __fmul2_rn(ly, m2);
  float2 q8 = __fmul2_rn(ly, m3);
  q8 = __ffma2_rn(lz, m2, q8);
  float2 q9 = __fmul2_rn(lz, m3);
  float2 q10 = __fmul2_rn(lx, m4);
  float2 q11 = __fmul2_rn(lx, m5);
  q11 = __ffma2_rn(ly, m4, q11);
  float2 q12 = __fmul2_rn(lx, m6);
  q12 = __ffma2_rn(lz, m4, q12);
  float2 q13 = __fmul2_rn(lx, m7);
  q13 = __ffma2_rn(ly, m5, q13);
  float2 q14 = __fmul2_rn(lx, m8);
  q14 = __ffma2_rn(ly, m6, q14);
  q14 = __ffma2_rn(lz, m5, q14);
  float2 q15 = __fmul2_rn(lx, m9);
  q15 = __ffma2_rn(lz, m6, q15);
  float2 q16 = __fmul2_rn(ly, m7);
  float2 q17 = __fmul2_rn(ly, m8);
  q17 = __ffma2_rn(lz, m7, q17);
  float2 q18 = __fmul2_rn(ly, m9);
  q18 = __ffma2_rn(lz, m8, q18);
  float2 q19 = __fmul2_rn(lz, m9);
  float2 S0, S1, G1x, G1y, G1z, S2, G2x, G2y, G2z, H2x, H2y, H2z, S3, G3x, H3x, G3y, H3y, G3z, H3z, S4, G4x, H4x, G4y, H4y, G4z, H4z;
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
    H2x = __fmul2_rn(b, q1);
  }
  { const float2 b = B[10];
    S2 = __ffma2_rn(b, m5, S2);
    G2x = __ffma2_rn(b, m2, G2x);
    H2x = __ffma2_rn(b, q2, H2x);
    G2y = __ffma2_rn(b, m1, G2y);
    H2y = __fmul2_rn(b, q1);
  }
  { const float2 b = B[11];
    S2 = __ffma2_rn(b, m6, S2);
    G2x = __ffma2_rn(b, m3, G2x);
    H2x = __ffma2_rn(b, q3, H2x);
    G2z = __ffma2_rn(b, m1, G2z);
    H2z = __fmul2_rn(b, q1);
  }
  { const float2 b = B[12];
    S2 = __ffma2_rn(b, m7, S2);
    G2y = __ffma2_rn(b, m2, G2y);
    H2y = __ffma2_rn(b, q2, H2y);
  }
  { const float2 b = B[13];
    S2 = __ffma2_rn(b, m8, S2);
    G2y = __ffma2_rn(b, m3, G2y);
    H2y = __ffma2_rn(b, q3, H2y);
    G2z = __ffma2_rn(b, m2, G2z);
    H2z = __ffma2_rn(b, q2, H2z);
  }
  { const float2 b = B[14];
    S2 = __ffma2_rn(b, m9, S2);
    G2z = __ffma2_rn(b, m3, G2z);
    H2z = __ffma2_rn(b, q3, H2z);
  }
  { const float2 b = B[15];
    S3 = __fmul2_rn(b, m4);
    G3x = __fmul2_rn(b, m1);
    H3x = __fmul2_rn(b, q1);
  }
  { const float2 b = B[16];
    S3 = __ffma2_rn(b, m5, S3);
    G3x = __ffma2_rn(b, m2, G3x);
    H3x = __ffma2_rn(b, q2, H3x);
    G3y = __fmul2_rn(b, m1);
    H3y = __fmul2_rn(b, q1);
  }
  { const float2 b = B[17];
    S3 = __ffma2_rn(b, m6, S3);
    G3x = __ffma2_rn(b, m3, G3x);
    H3x = __ffma2_rn(b, q3, H3x);
    G3z = __fmul2_rn(b, m1);
    H3z = __fmul2_rn(b, q1);
  }
  { const float2 b = B[18];
    S3 = __ffma2_rn(b, m7, S3);
    G3y = __ffma2_rn(b, m2, G3y);
    H3y = __ffma2_rn(b, q2, H3y);
  }
  { const float2 b = B[19];
    S3 = __ffma2_rn(b, m8, S3);
    G3y = __ffma2_rn(b, m3, G3y);
    H3y = __ffma2_rn(b, q3, H3y);
    G3z = __ffma2_rn(b, m2, G3z);
    H3z = __ffma2_rn(b, q2, H3z);
  }
  { const float2 b = B[20];
    S3 = __ffma2_rn(b, m9, S3);
    G3z = __ffma2_rn(b, m3, G3z);
    H3z = __ffma2_rn(b, q3, H3z);
  }
  { const float2 b = B[21];
    S3 = __ffma2_rn(b, m10, S3);
    G3x = __ffma2_rn(b, m4, G3x);
    H3x = __ffma2_rn(b, q4, H3x);
  }
  { const float2 b = B[22];
    S3 = __ffma2_rn(b, m11, S3);
    G3x = __ffma2_rn(b, m5, G3x);
    H3x = __ffma2_rn(b, q5, H3x);
    G3y = __ffma2_rn(b, m4, G3y);
    H3y = __ffma2_rn(b, q4, H3y);
  }
  { const float2 b = B[23];
    S3 = __ffma2_rn(b, m12, S3);
    G3x = __ffma2_rn(b, m6, G3x);
    H3x = __ffma2_rn(b, q6, H3x);
    G3z = __ffma2_rn(b, m4, G3z);
    H3z = __ffma2_rn(b, q4, H3z);
  }
  { const float2 b = B[24];
    S3 = __ffma2_rn(b, m13, S3);
    G3x = __ffma2_rn(b, m7, G3x);
    H3x = __ffma2_rn(b, q7, H3x);
    G3y = __ffma2_rn(b, m5, G3y);
    H3y = __ffma2_rn(b, q5, H3y);
  }
  { const float2 b = B[25];
    S3 = __ffma2_rn(b, m14, S3);
    G3x = __ffma2_rn(b, m8, G3x);
    H3x = __ffma2_rn(b, q8, H3x);
    G3y = __ffma2_rn(b, m6, G3y);
    H3y = __ffma2_rn(b, q6, H3y);
    G3z = __ffma2_rn(b, m5, G3z);
    H3z = __ffma2_rn(b, q5, H3z);
  }
  { const float2 b = B[26];
    S3 = __ffma2_rn(b, m15, S3);
    G3x = __ffma2_rn(b, m9, G3x);
    H3x = __ffma2_rn(b, q9, H3x);
    G3z = __ffma2_rn(b, m6, G3z);
    H3z = __ffma2_rn(b, q6, H3z);
  }
  { const float2 b = B[27];
    S3 = __ffma2_rn(b, m16, S3);
    G3y = __ffma2_rn(b, m7, G3y);
    H3y = __ffma2_rn(b, q7, H3y);
  }
  { const float2 b = B[28];
    S3 = __ffma2_rn(b, m17, S3);
    G3y = __ffma2_rn(b, m8, G3y);
    H3y = __ffma2_rn(b, q8, H3y);
    G3z = __ffma2_rn(b, m7, G3z);
    H3z = __ffma2_rn(b, q7, H3z);
  }
  { const float2 b = B[29];
    S3 = __ffma2_rn(b, m18, S3);
    G3y = __ffma2_rn(b, m9, G3y);
    H3y = __ffma2_rn(b, q9, H3y);
    G3z = __ffma2_rn(b, m8, G3z);
    H3z = __ffma2_rn(b, q8, H3z);
  }
  { const float2 b = B[30];
    S3 = __ffma2_rn(b, m19, S3);
    G3z = __ffma2_rn(b, m9, G3z);
    H3z = __ffma2_rn(b, q9, H3z);
  }
  { const float2 b = B[31];
    S4 = __fmul2_rn(b, m20);
    G4x = __fmul2_rn(b, m10);
    H4x = __fmul2_rn(b, q10);
  }
  { const float2 b = B[32];
    S4 = __ffma2_rn(b, m21, S4);
    G4x = __ffma2_rn(b, m11, G4x);
    H4x = __ffma2_rn(b, q11, H4x);
    G4y = __fmul2_rn(b, m10);
    H4y = __fmul2_rn(b, q10);
  }
  { const float2 b = B[33];
    S4 = __ffma2_rn(b, m22, S4);
    G4x = __ffma2_rn(b, m12, G4x);
    H4x = __ffma2_rn(b, q12, H4x);
    G4z = __fmul2_rn(b, m10);
    H4z = __fmul2_rn(b, q10);
  }
  { const float2 b = B[34];
    S4 = __ffma2_rn(b, m23, S4);
    G4x = __ffma2_rn(b, m13, G4x);
    H4x = __ffma2_rn(b, q13, H4x);
    G4y = __ffma2_rn(b, m11, G4y);
    H4y = __ffma2_rn(b, q11, H4y);
  }
  { const float2 b = B[35];
    S4 = __ffma2_rn(b, m24, S4);
    G4x = __ffma2_rn(b, m14, G4x);
    H4x = __ffma2_rn(b, q14, H4x);
    G4y = __ffma2_rn(b, m12, G4y);
    H4y = __ffma2_rn(b, q12, H4y);
    G4z = __ffma2_rn(b, m11, G4z);
    H4z = __ffma2_rn(b, q11, H4z);
  }
  { const float2 b = B[36];
    S4 = __ffma2_rn(b, m25, S4);
    G4x = __ffma2_rn(b, m15, G4x);
    H4x = __ffma2_rn(b, q15, H4x);
    G4z = __ffma2_rn(b, m12, G4z);
    H4z = __ffma2_rn(b, q12, H4z);
  }
  { const float2 b = B[37];
    S4 = __ffma2_rn(b, m26, S4);
    G4x = __ffma2_rn(b, m16, G4x);
    H4x = __ffma2_rn(b, q16, H4x);
    G4y = __ffma2_rn(b, m13, G4y);
    H4y = __ffma2_rn(b, q13, H4y);
  }
  { const float2 b = B[38];
    S4 = __ffma2_rn(b, m27, S4);
    G4x = __ffma2_rn(b, m17, G4x);
    H4x = __ffma2_rn(b, q17, H4x);
    G4y = __ffma2_rn(b, m14, G4y);
    H4y = __ffma2_rn(b, q14, H4y);
    G4z = __ffma2_rn(b, m13, G4z);
    H4z = __ffma2_rn(b, q13, H4z);
  }
  { const float2 b = B[39];
    S4 = __ffma2_rn(b, m28, S4);
    G4x = __ffma2_rn(b, m18, G4x);
    H4x = __ffma2_rn(b, q18, H4x);
    G4y = __ffma2_rn(b, m15, G4y);
    H4y = __ffma2_rn(b, q15, H4y);
    G4z = __ffma2_rn(b, m14, G4z);
    H4z = __ffma2_rn(b, q14, H4z);
  }
  { const float2 b = B[40];
    S4 = __ffma2_rn(b, m29, S4);
    G4x = __ffma2_rn(b, m19, G4x);
    H4x = __ffma2_rn(b, q19, H4x);
    G4z = __ffma2_rn(b, m15, G4z);
    H4z = __ffma2_rn(b, q15, H4z);
  }
  { const float2 b = B[41];
    S4 = __ffma2_rn(b, m30, S4);
    G4y = __ffma2_rn(b, m16, G4y);
    H4y = __ffma2_rn(b, q16, H4y);
  }
  { const float2 b = B[42];
    S4 = __ffma2_rn(b, m31, S4);
    G4y = __ffma2_rn(b, m17, G4y);
    H4y = __ffma2_rn(b, q17, H4y);
    G4z = __ffma2_rn(b, m16, G4z);
    H4z = __ffma2_rn(b, q16, H4z);
  }
  { const float2 b = B[43];
    S4 = __ffma2_rn(b, m32, S4);
    G4y = __ffma2_rn(b, m18, G4y);
    H4y = __ffma2_rn(b, q18, H4y);
    G4z = __ffma2_rn(b, m17, G4z);
    H4z = __ffma2_rn(b, q17, H4z);
  }
  { const float2 b = B[44];
    S4 = __ffma2_rn(b, m33, S4);
    G4y = __ffma2_rn(b, m19, G4y);
    H4y = __ffma2_rn(b, q19, H4y);
    G4z = __ffma2_rn(b, m18, G4z);
    H4z = __ffma2_rn(b, q18, H4z);
  }
  { const float2 b = B[45];
    S4 = __ffma2_rn(b, m34, S4);
    G4z = __ffma2_rn(b, m19, G4z);
    H4z = __ffma2_rn(b, q19, H4z);
  }
  const float2 rl = __ffma2_rn(Rx, lx, __ffma2_rn(Ry, ly, __fmul2_rn(Rz, lz)));
  float2 ax = ox, ay = oy, az = oz;
  { const float2 a1 = __fmul2_rn(F1, S0);
    const float2 c1 = __fmul2_rn(__fmul2_rn(F2, S0), rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, ax));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, ay));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, az));
  }
  { const float2 a1 = __fmul2_rn(F2, S1);
    const float2 gl = __ffma2_rn(G1x, lx, __ffma2_rn(G1y, ly, __fmul2_rn(G1z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F3, S1), rl, __fmul2_rn(F2, gl));
    const float2 c2 = __fmul2_rn(F2, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G1x, ax)));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G1y, ay)));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G1z, az)));
  }
  { const float2 a1 = __fmul2_rn(F3, S2);
    const float2 gl = __ffma2_rn(G2x, lx, __ffma2_rn(G2y, ly, __fmul2_rn(G2z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F4, S2), rl, __fmul2_rn(F3, gl));
    const float2 c2 = __fmul2_rn(F3, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G2x, __ffma2_rn(F2, H2x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G2y, __ffma2_rn(F2, H2y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G2z, __ffma2_rn(F2, H2z, az))));
  }
  { const float2 a1 = __fmul2_rn(F4, S3);
    const float2 gl = __ffma2_rn(G3x, lx, __ffma2_rn(G3y, ly, __fmul2_rn(G3z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F5, S3), rl, __fmul2_rn(F4, gl));
    const float2 c2 = __fmul2_rn(F4, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G3x, __ffma2_rn(F3, H3x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G3y, __ffma2_rn(F3, H3y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G3z, __ffma2_rn(F3, H3z, az))));
  }
  { const float2 a1 = __fmul2_rn(F5, S4);
    const float2 gl = __ffma2_rn(G4x, lx, __ffma2_rn(G4y, ly, __fmul2_rn(G4z, lz)));
    const float2 c1 = __ffma2_rn(__fmul2_rn(F6, S4), rl, __fmul2_rn(F5, gl));
    const float2 c2 = __fmul2_rn(F5, rl);
    ax = __ffma2_rn(a1, lx, __ffma2_rn(Rx, c1, __ffma2_rn(c2, G4x, __ffma2_rn(F4, H4x, ax))));
    ay = __ffma2_rn(a1, ly, __ffma2_rn(Ry, c1, __ffma2_rn(c2, G4y, __ffma2_rn(F4, H4y, ay))));
    az = __ffma2_rn(a1, lz, __ffma2_rn(Rz, c1, __ffma2_rn(c2, G4z, __ffma2_rn(F4, H4z, az))));
  }
  ox = ax;
  oy = ay;
  oz = az;
}

template <typename T>
__device__ __forceinline__ void m2p_adj_src_p4(T Rx, T Ry, T Rz, T eps2, T lx, T ly, T lz,
                                         T* __restrict__ nu) {
  const T s = fma(Rx, Rx, fma(Ry, Ry, fma(Rz, Rz, eps2)));
  const T F0 = nbody_rsqrt(s);
  const T is = F0 * F0;
  const T F1 = F0 * (T(-1) * is);
  const T F2 = F1 * (T(-3) * is);
  const T F3 = F2 * (T(-5) * is);
  const T F4 = F3 * (T(-7) * is);
  const T F5 = F4 * (T(-9) * is);
  const T r0 = T(1);
  const T r1 = Rx;
  const T r2 = Ry;
  const T r3 = Rz;
  const T r4 = r1 * Rx;
  const T r5 = r2 * Rx;
  const T r6 = r3 * Rx;
  const T r7 = r2 * Ry;
  const T r8 = r3 * Ry;
  const T r9 = r3 * Rz;
  const T r10 = r4 * Rx;
  const T r11 = r5 * Rx;
  const T r12 = r6 * Rx;
  const T r13 = r7 * Rx;
  const T r14 = r8 * Rx;
  const T r15 = r9 * Rx;
  const T r16 = r7 * Ry;
  const T r17 = r8 * Ry;
  const T r18 = r9 * Ry;
  const T r19 = r9 * Rz;
  const T r20 = r10 * Rx;
  const T r21 = r11 * Rx;
  const T r22 = r12 * Rx;
  const T r23 = r13 * Rx;
  const T r24 = r14 * Rx;
  const T r25 = r15 * Rx;
  const T r26 = r16 * Rx;
  const T r27 = r17 * Rx;
  const T r28 = r18 * Rx;
  const T r29 = r19 * Rx;
  const T r30 = r16 * Ry;
  const T r31 = r17 * Ry;
  const T r32 = r18 * Ry;
  const T r33 = r19 * Ry;
  const T r34 = r19 * Rz;
  const T E0 = F1 * (r0);
  const T E1 = F2 * (r1);
  const T E2 = F2 * (r2);
  const T E3 = F2 * (r3);
  const T E4 = fma(F3, r4, F2 * (r0));
  const T E5 = F3 * (r5);
  const T E6 = F3 * (r6);
  const T E7 = fma(F3, r7, F2 * (r0));
  const T E8 = F3 * (r8);
  const T E9 = fma(F3, r9, F2 * (r0));
  const T E10 = fma(F4, r10, F3 * (r1 * T(3)));
  const T E11 = fma(F4, r11, F3 * (r2));
  const T E12 = fma(F4, r12, F3 * (r3));
  const T E13 = fma(F4, r13, F3 * (r1));
  const T E14 = F4 * (r14);
  const T E15 = fma(F4, r15, F3 * (r1));
  const T E16 = fma(F4, r16, F3 * (r2 * T(3)));
  const T E17 = fma(F4, r17, F3 * (r3));
  const T E18 = fma(F4, r18, F3 * (r2));
  const T E19 = fma(F4, r19, F3 * (r3 * T(3)));
  const T E20 = fma(F5, r20, fma(F4, r4 * T(6), F3 * (r0 * T(3))));
  const T E21 = fma(F5, r21, F4 * (r5 * T(3)));
  const T E22 = fma(F5, r22, F4 * (r6 * T(3)));
  const T E23 = fma(F5, r23, fma(F4, fma(r7, T(1), r4), F3 * (r0)));
  const T E24 = fma(F5, r24, F4 * (r8));
  const T E25 = fma(F5, r25, fma(F4, fma(r9, T(1), r4), F3 * (r0)));
  const T E26 = fma(F5, r26, F4 * (r5 * T(3)));
  const T E27 = fma(F5, r27, F4 * (r6));
  const T E28 = fma(F5, r28, F4 * (r5));
  const T E29 = fma(F5, r29, F4 * (r6 * T(3)));
  const T E30 = fma(F5, r30, fma(F4, r7 * T(6), F3 * (r0 * T(3))));
  const T E31 = fma(F5, r31, F4 * (r8 * T(3)));
  const T E32 = fma(F5, r32, fma(F4, fma(r9, T(1), r7), F3 * (r0)));
  const T E33 = fma(F5, r33, F4 * (r8 * T(3)));
  const T E34 = fma(F5, r34, fma(F4, r9 * T(6), F3 * (r0 * T(3))));
  const T rl = fma(Rx, lx, fma(Ry, ly, Rz * lz));
  nu[0] = fma(rl, E0, nu[0]);
  nu[1] = fma(lx, E0, fma(rl, E1, nu[1]));
  nu[2] = fma(ly, E0, fma(rl, E2, nu[2]));
  nu[3] = fma(lz, E0, fma(rl, E3, nu[3]));
  nu[4] = fma((lx * T(2)), E1, fma(rl, E4, nu[4]));
  nu[5] = fma(ly, E1, fma(lx, E2, fma(rl, E5, nu[5])));
  nu[6] = fma(lz, E1, fma(lx, E3, fma(rl, E6, nu[6])));
  nu[7] = fma((ly * T(2)), E2, fma(rl, E7, nu[7]));
  nu[8] = fma(lz, E2, fma(ly, E3, fma(rl, E8, nu[8])));
  nu[9] = fma((lz * T(2)), E3, fma(rl, E9, nu[9]));
  nu[10] = fma((lx * T(3)), E4, fma(rl, E10, nu[10]));
  nu[11] = fma(ly, E4, fma((lx * T(2)), E5, fma(rl, E11, nu[11])));
  nu[12] = fma(lz, E4, fma((lx * T(2)), E6, fma(rl, E12, nu[12])));
  nu[13] = fma((ly * T(2)), E5, fma(lx, E7, fma(rl, E13, nu[13])));
  nu[14] = fma(lz, E5, fma(ly, E6, fma(lx, E8, fma(rl, E14, nu[14]))));
  nu[15] = fma((lz * T(2)), E6, fma(lx, E9, fma(rl, E15, nu[15])));
  nu[16] = fma((ly * T(3)), E7, fma(rl, E16, nu[16]));
  nu[17] = fma(lz, E7, fma((ly * T(2)), E8, fma(rl, E17, nu[17])));
  nu[18] = fma((lz * T(2)), E8, fma(ly, E9, fma(rl, E18, nu[18])));
  nu[19] = fma((lz * T(3)), E9, fma(rl, E19, nu[19]));
  nu[20] = fma((lx * T(4)), E10, fma(rl, E20, nu[20]));
  nu[21] = fma(ly, E10, fma((lx * T(3)), E11, fma(rl, E21, nu[21])));
  nu[22] = fma(lz, E10, fma((lx * T(3)), E12, fma(rl, E22, nu[22])));
  nu[23] = fma((ly * T(2)), E11, fma((lx * T(2)), E13, fma(rl, E23, nu[23])));
  nu[24] = fma(lz, E11, fma(ly, E12, fma((lx * T(2)), E14, fma(rl, E24, nu[24]))));
  nu[25] = fma((lz * T(2)), E12, fma((lx * T(2)), E15, fma(rl, E25, nu[25])));
  nu[26] = fma((ly * T(3)), E13, fma(lx, E16, fma(rl, E26, nu[26])));
  nu[27] = fma(lz, E13, fma((ly * T(2)), E14, fma(lx, E17, fma(rl, E27, nu[27]))));
  nu[28] = fma((lz * T(2)), E14, fma(ly, E15, fma(lx, E18, fma(rl, E28, nu[28]))));
  nu[29] = fma((lz * T(3)), E15, fma(lx, E19, fma(rl, E29, nu[29])));
  nu[30] = fma((ly * T(4)), E16, fma(rl, E30, nu[30]));
  nu[31] = fma(lz, E16, fma((ly * T(3)), E17, fma(rl, E31, nu[31])));
  nu[32] = fma((lz * T(2)), E17, fma((ly * T(2)), E18, fma(rl, E32, nu[32])));
  nu[33] = fma((lz * T(3)), E18, fma(ly, E19, fma(rl, E33, nu[33])));
  nu[34] = fma((lz * T(4)), E19, fma(rl, E34, nu[34]));
}

__device__ __forceinline__ void m2m_adj_acc_p4(const double* __restrict__ nup, double sx, double sy, double sz, double* __restrict__ nuc) {
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
  nuc[0] = fma(w34, nup[34], fma(w33, nup[33], fma(w32, nup[32], fma(w31, nup[31], fma(w30, nup[30], fma(w29, nup[29], fma(w28, nup[28], fma(w27, nup[27], fma(w26, nup[26], fma(w25, nup[25], fma(w24, nup[24], fma(w23, nup[23], fma(w22, nup[22], fma(w21, nup[21], fma(w20, nup[20], fma(w19, nup[19], fma(w18, nup[18], fma(w17, nup[17], fma(w16, nup[16], fma(w15, nup[15], fma(w14, nup[14], fma(w13, nup[13], fma(w12, nup[12], fma(w11, nup[11], fma(w10, nup[10], fma(w9, nup[9], fma(w8, nup[8], fma(w7, nup[7], fma(w6, nup[6], fma(w5, nup[5], fma(w4, nup[4], fma(w3, nup[3], fma(w2, nup[2], fma(w1, nup[1], fma(w0, nup[0], nuc[0])))))))))))))))))))))))))))))))))));
  nuc[1] = fma(w19, nup[29], fma(w18, nup[28], fma(w17, nup[27], fma(w16, nup[26], fma(w15 * 2.0, nup[25], fma(w14 * 2.0, nup[24], fma(w13 * 2.0, nup[23], fma(w12 * 3.0, nup[22], fma(w11 * 3.0, nup[21], fma(w10 * 4.0, nup[20], fma(w9, nup[15], fma(w8, nup[14], fma(w7, nup[13], fma(w6 * 2.0, nup[12], fma(w5 * 2.0, nup[11], fma(w4 * 3.0, nup[10], fma(w3, nup[6], fma(w2, nup[5], fma(w1 * 2.0, nup[4], fma(w0, nup[1], nuc[1]))))))))))))))))))));
  nuc[2] = fma(w19, nup[33], fma(w18 * 2.0, nup[32], fma(w17 * 3.0, nup[31], fma(w16 * 4.0, nup[30], fma(w15, nup[28], fma(w14 * 2.0, nup[27], fma(w13 * 3.0, nup[26], fma(w12, nup[24], fma(w11 * 2.0, nup[23], fma(w10, nup[21], fma(w9, nup[18], fma(w8 * 2.0, nup[17], fma(w7 * 3.0, nup[16], fma(w6, nup[14], fma(w5 * 2.0, nup[13], fma(w4, nup[11], fma(w3, nup[8], fma(w2 * 2.0, nup[7], fma(w1, nup[5], fma(w0, nup[2], nuc[2]))))))))))))))))))));
  nuc[3] = fma(w19 * 4.0, nup[34], fma(w18 * 3.0, nup[33], fma(w17 * 2.0, nup[32], fma(w16, nup[31], fma(w15 * 3.0, nup[29], fma(w14 * 2.0, nup[28], fma(w13, nup[27], fma(w12 * 2.0, nup[25], fma(w11, nup[24], fma(w10, nup[22], fma(w9 * 3.0, nup[19], fma(w8 * 2.0, nup[18], fma(w7, nup[17], fma(w6 * 2.0, nup[15], fma(w5, nup[14], fma(w4, nup[12], fma(w3 * 2.0, nup[9], fma(w2, nup[8], fma(w1, nup[6], fma(w0, nup[3], nuc[3]))))))))))))))))))));
  nuc[4] = fma(w9, nup[25], fma(w8, nup[24], fma(w7, nup[23], fma(w6 * 3.0, nup[22], fma(w5 * 3.0, nup[21], fma(w4 * 6.0, nup[20], fma(w3, nup[12], fma(w2, nup[11], fma(w1 * 3.0, nup[10], fma(w0, nup[4], nuc[4]))))))))));
  nuc[5] = fma(w9, nup[28], fma(w8 * 2.0, nup[27], fma(w7 * 3.0, nup[26], fma(w6 * 2.0, nup[24], fma(w5 * 4.0, nup[23], fma(w4 * 3.0, nup[21], fma(w3, nup[14], fma(w2 * 2.0, nup[13], fma(w1 * 2.0, nup[11], fma(w0, nup[5], nuc[5]))))))))));
  nuc[6] = fma(w9 * 3.0, nup[29], fma(w8 * 2.0, nup[28], fma(w7, nup[27], fma(w6 * 4.0, nup[25], fma(w5 * 2.0, nup[24], fma(w4 * 3.0, nup[22], fma(w3 * 2.0, nup[15], fma(w2, nup[14], fma(w1 * 2.0, nup[12], fma(w0, nup[6], nuc[6]))))))))));
  nuc[7] = fma(w9, nup[32], fma(w8 * 3.0, nup[31], fma(w7 * 6.0, nup[30], fma(w6, nup[27], fma(w5 * 3.0, nup[26], fma(w4, nup[23], fma(w3, nup[17], fma(w2 * 3.0, nup[16], fma(w1, nup[13], fma(w0, nup[7], nuc[7]))))))))));
  nuc[8] = fma(w9 * 3.0, nup[33], fma(w8 * 4.0, nup[32], fma(w7 * 3.0, nup[31], fma(w6 * 2.0, nup[28], fma(w5 * 2.0, nup[27], fma(w4, nup[24], fma(w3 * 2.0, nup[18], fma(w2 * 2.0, nup[17], fma(w1, nup[14], fma(w0, nup[8], nuc[8]))))))))));
  nuc[9] = fma(w9 * 6.0, nup[34], fma(w8 * 3.0, nup[33], fma(w7, nup[32], fma(w6 * 3.0, nup[29], fma(w5, nup[28], fma(w4, nup[25], fma(w3 * 3.0, nup[19], fma(w2, nup[18], fma(w1, nup[15], fma(w0, nup[9], nuc[9]))))))))));
  nuc[10] = fma(w3, nup[22], fma(w2, nup[21], fma(w1 * 4.0, nup[20], fma(w0, nup[10], nuc[10]))));
  nuc[11] = fma(w3, nup[24], fma(w2 * 2.0, nup[23], fma(w1 * 3.0, nup[21], fma(w0, nup[11], nuc[11]))));
  nuc[12] = fma(w3 * 2.0, nup[25], fma(w2, nup[24], fma(w1 * 3.0, nup[22], fma(w0, nup[12], nuc[12]))));
  nuc[13] = fma(w3, nup[27], fma(w2 * 3.0, nup[26], fma(w1 * 2.0, nup[23], fma(w0, nup[13], nuc[13]))));
  nuc[14] = fma(w3 * 2.0, nup[28], fma(w2 * 2.0, nup[27], fma(w1 * 2.0, nup[24], fma(w0, nup[14], nuc[14]))));
  nuc[15] = fma(w3 * 3.0, nup[29], fma(w2, nup[28], fma(w1 * 2.0, nup[25], fma(w0, nup[15], nuc[15]))));
  nuc[16] = fma(w3, nup[31], fma(w2 * 4.0, nup[30], fma(w1, nup[26], fma(w0, nup[16], nuc[16]))));
  nuc[17] = fma(w3 * 2.0, nup[32], fma(w2 * 3.0, nup[31], fma(w1, nup[27], fma(w0, nup[17], nuc[17]))));
  nuc[18] = fma(w3 * 3.0, nup[33], fma(w2 * 2.0, nup[32], fma(w1, nup[28], fma(w0, nup[18], nuc[18]))));
  nuc[19] = fma(w3 * 4.0, nup[34], fma(w2, nup[33], fma(w1, nup[29], fma(w0, nup[19], nuc[19]))));
  nuc[20] = fma(w0, nup[20], nuc[20]);
  nuc[21] = fma(w0, nup[21], nuc[21]);
  nuc[22] = fma(w0, nup[22], nuc[22]);
  nuc[23] = fma(w0, nup[23], nuc[23]);
  nuc[24] = fma(w0, nup[24], nuc[24]);
  nuc[25] = fma(w0, nup[25], nuc[25]);
  nuc[26] = fma(w0, nup[26], nuc[26]);
  nuc[27] = fma(w0, nup[27], nuc[27]);
  nuc[28] = fma(w0, nup[28], nuc[28]);
  nuc[29] = fma(w0, nup[29], nuc[29]);
  nuc[30] = fma(w0, nup[30], nuc[30]);
  nuc[31] = fma(w0, nup[31], nuc[31]);
  nuc[32] = fma(w0, nup[32], nuc[32]);
  nuc[33] = fma(w0, nup[33], nuc[33]);
  nuc[34] = fma(w0, nup[34], nuc[34]);
}

__device__ __forceinline__ void p2m_adj_p4(double m, double dx, double dy, double dz, const double* __restrict__ nu, double& gx, double& gy, double& gz) {
  const double q0 = 1.0;
  const double q1 = q0 * dx;
  const double q2 = q0 * dy;
  const double q3 = q0 * dz;
  const double q4 = q1 * dx;
  const double q5 = q2 * dx;
  const double q6 = q3 * dx;
  const double q7 = q2 * dy;
  const double q8 = q3 * dy;
  const double q9 = q3 * dz;
  const double q10 = q4 * dx;
  const double q11 = q5 * dx;
  const double q12 = q6 * dx;
  const double q13 = q7 * dx;
  const double q14 = q8 * dx;
  const double q15 = q9 * dx;
  const double q16 = q7 * dy;
  const double q17 = q8 * dy;
  const double q18 = q9 * dy;
  const double q19 = q9 * dz;
  gx = fma(m, fma(nu[29], q19, fma(nu[28], q18, fma(nu[27], q17, fma(nu[26], q16, fma(nu[25] * 2.0, q15, fma(nu[24] * 2.0, q14, fma(nu[23] * 2.0, q13, fma(nu[22] * 3.0, q12, fma(nu[21] * 3.0, q11, fma(nu[20] * 4.0, q10, fma(nu[15], q9, fma(nu[14], q8, fma(nu[13], q7, fma(nu[12] * 2.0, q6, fma(nu[11] * 2.0, q5, fma(nu[10] * 3.0, q4, fma(nu[6], q3, fma(nu[5], q2, fma(nu[4] * 2.0, q1, fma(nu[1], q0, 0.0)))))))))))))))))))), gx);
  gy = fma(m, fma(nu[33], q19, fma(nu[32] * 2.0, q18, fma(nu[31] * 3.0, q17, fma(nu[30] * 4.0, q16, fma(nu[28], q15, fma(nu[27] * 2.0, q14, fma(nu[26] * 3.0, q13, fma(nu[24], q12, fma(nu[23] * 2.0, q11, fma(nu[21], q10, fma(nu[18], q9, fma(nu[17] * 2.0, q8, fma(nu[16] * 3.0, q7, fma(nu[14], q6, fma(nu[13] * 2.0, q5, fma(nu[11], q4, fma(nu[8], q3, fma(nu[7] * 2.0, q2, fma(nu[5], q1, fma(nu[2], q0, 0.0)))))))))))))))))))), gy);
  gz = fma(m, fma(nu[34] * 4.0, q19, fma(nu[33] * 3.0, q18, fma(nu[32] * 2.0, q17, fma(nu[31], q16, fma(nu[29] * 3.0, q15, fma(nu[28] * 2.0, q14, fma(nu[27], q13, fma(nu[25] * 2.0, q12, fma(nu[24], q11, fma(nu[22], q10, fma(nu[19] * 3.0, q9, fma(nu[18] * 2.0, q8, fma(nu[17], q7, fma(nu[15] * 2.0, q6, fma(nu[14], q5, fma(nu[12], q4, fma(nu[9] * 2.0, q3, fma(nu[8], q2, fma(nu[6], q1, fma(nu[3], q0, 0.0)))))))))))))))))))), gz);
}

template <typename T>
__device__ __forceinline__ void l2p_hess_pe1(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T q0 = T(1);
  ox = fma(-lz * q0, Lc[5], fma(-ly * q0, Lc[4], fma(-lx * q0, Lc[3], ox)));
  oy = fma(-lz * q0, Lc[7], fma(-ly * q0, Lc[6], fma(-lx * q0, Lc[4], oy)));
  oz = fma(-lz * q0, Lc[8], fma(-ly * q0, Lc[7], fma(-lx * q0, Lc[5], oz)));
}
template <typename T>
__device__ __forceinline__ void l2p_adj_pe1(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  Lbar[0] = fma(-lx, q0, Lbar[0]);
  Lbar[1] = fma(-ly, q0, Lbar[1]);
  Lbar[2] = fma(-lz, q0, Lbar[2]);
  Lbar[3] = fma(-lx, q1, Lbar[3]);
  Lbar[4] = fma(-ly, q1, fma(-lx, q2, Lbar[4]));
  Lbar[5] = fma(-lz, q1, fma(-lx, q3, Lbar[5]));
  Lbar[6] = fma(-ly, q2, Lbar[6]);
  Lbar[7] = fma(-lz, q2, fma(-ly, q3, Lbar[7]));
  Lbar[8] = fma(-lz, q3, Lbar[8]);
}
template <typename T>
__device__ __forceinline__ void m2l_adj_pe1(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {
  nu[0] = fma(T(1), fma(Lbar[8], D[9], fma(Lbar[7], D[8], fma(Lbar[6], D[7], fma(Lbar[5], D[6], fma(Lbar[4], D[5], fma(Lbar[3], D[4], fma(Lbar[2], D[3], fma(Lbar[1], D[2], Lbar[0] * D[1])))))))), nu[0]);
  nu[1] = fma(T(-1), fma(Lbar[2], D[6], fma(Lbar[1], D[5], Lbar[0] * D[4])), nu[1]);
  nu[2] = fma(T(-1), fma(Lbar[2], D[8], fma(Lbar[1], D[7], Lbar[0] * D[5])), nu[2]);
  nu[3] = fma(T(-1), fma(Lbar[2], D[9], fma(Lbar[1], D[8], Lbar[0] * D[6])), nu[3]);
}

template <typename T>
__device__ __forceinline__ void l2p_hess_pe2(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {
  const T q0 = T(1);
  const T q1 = q0 * (dx * T(1));
  const T q2 = q0 * (dy * T(1));
  const T q3 = q0 * (dz * T(1));
  ox = fma(-lz * q3, Lc[14], fma(-lz * q2, Lc[13], fma(-lz * q1, Lc[11], fma(-lz * q0, Lc[5], fma(-ly * q3, Lc[13], fma(-ly * q2, Lc[12], fma(-ly * q1, Lc[10], fma(-ly * q0, Lc[4], fma(-lx * q3, Lc[11], fma(-lx * q2, Lc[10], fma(-lx * q1, Lc[9], fma(-lx * q0, Lc[3], ox))))))))))));
  oy = fma(-lz * q3, Lc[17], fma(-lz * q2, Lc[16], fma(-lz * q1, Lc[13], fma(-lz * q0, Lc[7], fma(-ly * q3, Lc[16], fma(-ly * q2, Lc[15], fma(-ly * q1, Lc[12], fma(-ly * q0, Lc[6], fma(-lx * q3, Lc[13], fma(-lx * q2, Lc[12], fma(-lx * q1, Lc[10], fma(-lx * q0, Lc[4], oy))))))))))));
  oz = fma(-lz * q3, Lc[18], fma(-lz * q2, Lc[17], fma(-lz * q1, Lc[14], fma(-lz * q0, Lc[8], fma(-ly * q3, Lc[17], fma(-ly * q2, Lc[16], fma(-ly * q1, Lc[13], fma(-ly * q0, Lc[7], fma(-lx * q3, Lc[14], fma(-lx * q2, Lc[13], fma(-lx * q1, Lc[11], fma(-lx * q0, Lc[5], oz))))))))))));
}
template <typename T>
__device__ __forceinline__ void l2p_adj_pe2(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {
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
  Lbar[0] = fma(-lx, q0, Lbar[0]);
  Lbar[1] = fma(-ly, q0, Lbar[1]);
  Lbar[2] = fma(-lz, q0, Lbar[2]);
  Lbar[3] = fma(-lx, q1, Lbar[3]);
  Lbar[4] = fma(-ly, q1, fma(-lx, q2, Lbar[4]));
  Lbar[5] = fma(-lz, q1, fma(-lx, q3, Lbar[5]));
  Lbar[6] = fma(-ly, q2, Lbar[6]);
  Lbar[7] = fma(-lz, q2, fma(-ly, q3, Lbar[7]));
  Lbar[8] = fma(-lz, q3, Lbar[8]);
  Lbar[9] = fma(-lx, q4, Lbar[9]);
  Lbar[10] = fma(-ly, q4, fma(-lx, q5, Lbar[10]));
  Lbar[11] = fma(-lz, q4, fma(-lx, q6, Lbar[11]));
  Lbar[12] = fma(-ly, q5, fma(-lx, q7, Lbar[12]));
  Lbar[13] = fma(-lz, q5, fma(-ly, q6, fma(-lx, q8, Lbar[13])));
  Lbar[14] = fma(-lz, q6, fma(-lx, q9, Lbar[14]));
  Lbar[15] = fma(-ly, q7, Lbar[15]);
  Lbar[16] = fma(-lz, q7, fma(-ly, q8, Lbar[16]));
  Lbar[17] = fma(-lz, q8, fma(-ly, q9, Lbar[17]));
  Lbar[18] = fma(-lz, q9, Lbar[18]);
}
template <typename T>
__device__ __forceinline__ void m2l_adj_pe2(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {
  nu[0] = fma(T(1), fma(Lbar[18], D[19], fma(Lbar[17], D[18], fma(Lbar[16], D[17], fma(Lbar[15], D[16], fma(Lbar[14], D[15], fma(Lbar[13], D[14], fma(Lbar[12], D[13], fma(Lbar[11], D[12], fma(Lbar[10], D[11], fma(Lbar[9], D[10], fma(Lbar[8], D[9], fma(Lbar[7], D[8], fma(Lbar[6], D[7], fma(Lbar[5], D[6], fma(Lbar[4], D[5], fma(Lbar[3], D[4], fma(Lbar[2], D[3], fma(Lbar[1], D[2], Lbar[0] * D[1])))))))))))))))))), nu[0]);
  nu[1] = fma(T(-1), fma(Lbar[8], D[15], fma(Lbar[7], D[14], fma(Lbar[6], D[13], fma(Lbar[5], D[12], fma(Lbar[4], D[11], fma(Lbar[3], D[10], fma(Lbar[2], D[6], fma(Lbar[1], D[5], Lbar[0] * D[4])))))))), nu[1]);
  nu[2] = fma(T(-1), fma(Lbar[8], D[18], fma(Lbar[7], D[17], fma(Lbar[6], D[16], fma(Lbar[5], D[14], fma(Lbar[4], D[13], fma(Lbar[3], D[11], fma(Lbar[2], D[8], fma(Lbar[1], D[7], Lbar[0] * D[5])))))))), nu[2]);
  nu[3] = fma(T(-1), fma(Lbar[8], D[19], fma(Lbar[7], D[18], fma(Lbar[6], D[17], fma(Lbar[5], D[15], fma(Lbar[4], D[14], fma(Lbar[3], D[12], fma(Lbar[2], D[9], fma(Lbar[1], D[8], Lbar[0] * D[6])))))))), nu[3]);
  nu[4] = fma(T(0.5), fma(Lbar[2], D[12], fma(Lbar[1], D[11], Lbar[0] * D[10])), nu[4]);
  nu[5] = fma(T(1), fma(Lbar[2], D[14], fma(Lbar[1], D[13], Lbar[0] * D[11])), nu[5]);
  nu[6] = fma(T(1), fma(Lbar[2], D[15], fma(Lbar[1], D[14], Lbar[0] * D[12])), nu[6]);
  nu[7] = fma(T(0.5), fma(Lbar[2], D[17], fma(Lbar[1], D[16], Lbar[0] * D[13])), nu[7]);
  nu[8] = fma(T(1), fma(Lbar[2], D[18], fma(Lbar[1], D[17], Lbar[0] * D[14])), nu[8]);
  nu[9] = fma(T(0.5), fma(Lbar[2], D[19], fma(Lbar[1], D[18], Lbar[0] * D[15])), nu[9]);
}

template <typename T>
__device__ __forceinline__ void l2p_hess_pe3(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {
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
  ox = fma(-lz * q9, Lc[28], fma(-lz * q8, Lc[27], fma(-lz * q7, Lc[26], fma(-lz * q6, Lc[24], fma(-lz * q5, Lc[23], fma(-lz * q4, Lc[21], fma(-lz * q3, Lc[14], fma(-lz * q2, Lc[13], fma(-lz * q1, Lc[11], fma(-lz * q0, Lc[5], fma(-ly * q9, Lc[27], fma(-ly * q8, Lc[26], fma(-ly * q7, Lc[25], fma(-ly * q6, Lc[23], fma(-ly * q5, Lc[22], fma(-ly * q4, Lc[20], fma(-ly * q3, Lc[13], fma(-ly * q2, Lc[12], fma(-ly * q1, Lc[10], fma(-ly * q0, Lc[4], fma(-lx * q9, Lc[24], fma(-lx * q8, Lc[23], fma(-lx * q7, Lc[22], fma(-lx * q6, Lc[21], fma(-lx * q5, Lc[20], fma(-lx * q4, Lc[19], fma(-lx * q3, Lc[11], fma(-lx * q2, Lc[10], fma(-lx * q1, Lc[9], fma(-lx * q0, Lc[3], ox))))))))))))))))))))))))))))));
  oy = fma(-lz * q9, Lc[32], fma(-lz * q8, Lc[31], fma(-lz * q7, Lc[30], fma(-lz * q6, Lc[27], fma(-lz * q5, Lc[26], fma(-lz * q4, Lc[23], fma(-lz * q3, Lc[17], fma(-lz * q2, Lc[16], fma(-lz * q1, Lc[13], fma(-lz * q0, Lc[7], fma(-ly * q9, Lc[31], fma(-ly * q8, Lc[30], fma(-ly * q7, Lc[29], fma(-ly * q6, Lc[26], fma(-ly * q5, Lc[25], fma(-ly * q4, Lc[22], fma(-ly * q3, Lc[16], fma(-ly * q2, Lc[15], fma(-ly * q1, Lc[12], fma(-ly * q0, Lc[6], fma(-lx * q9, Lc[27], fma(-lx * q8, Lc[26], fma(-lx * q7, Lc[25], fma(-lx * q6, Lc[23], fma(-lx * q5, Lc[22], fma(-lx * q4, Lc[20], fma(-lx * q3, Lc[13], fma(-lx * q2, Lc[12], fma(-lx * q1, Lc[10], fma(-lx * q0, Lc[4], oy))))))))))))))))))))))))))))));
  oz = fma(-lz * q9, Lc[33], fma(-lz * q8, Lc[32], fma(-lz * q7, Lc[31], fma(-lz * q6, Lc[28], fma(-lz * q5, Lc[27], fma(-lz * q4, Lc[24], fma(-lz * q3, Lc[18], fma(-lz * q2, Lc[17], fma(-lz * q1, Lc[14], fma(-lz * q0, Lc[8], fma(-ly * q9, Lc[32], fma(-ly * q8, Lc[31], fma(-ly * q7, Lc[30], fma(-ly * q6, Lc[27], fma(-ly * q5, Lc[26], fma(-ly * q4, Lc[23], fma(-ly * q3, Lc[17], fma(-ly * q2, Lc[16], fma(-ly * q1, Lc[13], fma(-ly * q0, Lc[7], fma(-lx * q9, Lc[28], fma(-lx * q8, Lc[27], fma(-lx * q7, Lc[26], fma(-lx * q6, Lc[24], fma(-lx * q5, Lc[23], fma(-lx * q4, Lc[21], fma(-lx * q3, Lc[14], fma(-lx * q2, Lc[13], fma(-lx * q1, Lc[11], fma(-lx * q0, Lc[5], oz))))))))))))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ void l2p_adj_pe3(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {
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
  Lbar[0] = fma(-lx, q0, Lbar[0]);
  Lbar[1] = fma(-ly, q0, Lbar[1]);
  Lbar[2] = fma(-lz, q0, Lbar[2]);
  Lbar[3] = fma(-lx, q1, Lbar[3]);
  Lbar[4] = fma(-ly, q1, fma(-lx, q2, Lbar[4]));
  Lbar[5] = fma(-lz, q1, fma(-lx, q3, Lbar[5]));
  Lbar[6] = fma(-ly, q2, Lbar[6]);
  Lbar[7] = fma(-lz, q2, fma(-ly, q3, Lbar[7]));
  Lbar[8] = fma(-lz, q3, Lbar[8]);
  Lbar[9] = fma(-lx, q4, Lbar[9]);
  Lbar[10] = fma(-ly, q4, fma(-lx, q5, Lbar[10]));
  Lbar[11] = fma(-lz, q4, fma(-lx, q6, Lbar[11]));
  Lbar[12] = fma(-ly, q5, fma(-lx, q7, Lbar[12]));
  Lbar[13] = fma(-lz, q5, fma(-ly, q6, fma(-lx, q8, Lbar[13])));
  Lbar[14] = fma(-lz, q6, fma(-lx, q9, Lbar[14]));
  Lbar[15] = fma(-ly, q7, Lbar[15]);
  Lbar[16] = fma(-lz, q7, fma(-ly, q8, Lbar[16]));
  Lbar[17] = fma(-lz, q8, fma(-ly, q9, Lbar[17]));
  Lbar[18] = fma(-lz, q9, Lbar[18]);
  Lbar[19] = fma(-lx, q10, Lbar[19]);
  Lbar[20] = fma(-ly, q10, fma(-lx, q11, Lbar[20]));
  Lbar[21] = fma(-lz, q10, fma(-lx, q12, Lbar[21]));
  Lbar[22] = fma(-ly, q11, fma(-lx, q13, Lbar[22]));
  Lbar[23] = fma(-lz, q11, fma(-ly, q12, fma(-lx, q14, Lbar[23])));
  Lbar[24] = fma(-lz, q12, fma(-lx, q15, Lbar[24]));
  Lbar[25] = fma(-ly, q13, fma(-lx, q16, Lbar[25]));
  Lbar[26] = fma(-lz, q13, fma(-ly, q14, fma(-lx, q17, Lbar[26])));
  Lbar[27] = fma(-lz, q14, fma(-ly, q15, fma(-lx, q18, Lbar[27])));
  Lbar[28] = fma(-lz, q15, fma(-lx, q19, Lbar[28]));
  Lbar[29] = fma(-ly, q16, Lbar[29]);
  Lbar[30] = fma(-lz, q16, fma(-ly, q17, Lbar[30]));
  Lbar[31] = fma(-lz, q17, fma(-ly, q18, Lbar[31]));
  Lbar[32] = fma(-lz, q18, fma(-ly, q19, Lbar[32]));
  Lbar[33] = fma(-lz, q19, Lbar[33]);
}
template <typename T>
__device__ __forceinline__ void m2l_adj_pe3(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {
  nu[0] = fma(T(1), fma(Lbar[33], D[34], fma(Lbar[32], D[33], fma(Lbar[31], D[32], fma(Lbar[30], D[31], fma(Lbar[29], D[30], fma(Lbar[28], D[29], fma(Lbar[27], D[28], fma(Lbar[26], D[27], fma(Lbar[25], D[26], fma(Lbar[24], D[25], fma(Lbar[23], D[24], fma(Lbar[22], D[23], fma(Lbar[21], D[22], fma(Lbar[20], D[21], fma(Lbar[19], D[20], fma(Lbar[18], D[19], fma(Lbar[17], D[18], fma(Lbar[16], D[17], fma(Lbar[15], D[16], fma(Lbar[14], D[15], fma(Lbar[13], D[14], fma(Lbar[12], D[13], fma(Lbar[11], D[12], fma(Lbar[10], D[11], fma(Lbar[9], D[10], fma(Lbar[8], D[9], fma(Lbar[7], D[8], fma(Lbar[6], D[7], fma(Lbar[5], D[6], fma(Lbar[4], D[5], fma(Lbar[3], D[4], fma(Lbar[2], D[3], fma(Lbar[1], D[2], Lbar[0] * D[1]))))))))))))))))))))))))))))))))), nu[0]);
  nu[1] = fma(T(-1), fma(Lbar[18], D[29], fma(Lbar[17], D[28], fma(Lbar[16], D[27], fma(Lbar[15], D[26], fma(Lbar[14], D[25], fma(Lbar[13], D[24], fma(Lbar[12], D[23], fma(Lbar[11], D[22], fma(Lbar[10], D[21], fma(Lbar[9], D[20], fma(Lbar[8], D[15], fma(Lbar[7], D[14], fma(Lbar[6], D[13], fma(Lbar[5], D[12], fma(Lbar[4], D[11], fma(Lbar[3], D[10], fma(Lbar[2], D[6], fma(Lbar[1], D[5], Lbar[0] * D[4])))))))))))))))))), nu[1]);
  nu[2] = fma(T(-1), fma(Lbar[18], D[33], fma(Lbar[17], D[32], fma(Lbar[16], D[31], fma(Lbar[15], D[30], fma(Lbar[14], D[28], fma(Lbar[13], D[27], fma(Lbar[12], D[26], fma(Lbar[11], D[24], fma(Lbar[10], D[23], fma(Lbar[9], D[21], fma(Lbar[8], D[18], fma(Lbar[7], D[17], fma(Lbar[6], D[16], fma(Lbar[5], D[14], fma(Lbar[4], D[13], fma(Lbar[3], D[11], fma(Lbar[2], D[8], fma(Lbar[1], D[7], Lbar[0] * D[5])))))))))))))))))), nu[2]);
  nu[3] = fma(T(-1), fma(Lbar[18], D[34], fma(Lbar[17], D[33], fma(Lbar[16], D[32], fma(Lbar[15], D[31], fma(Lbar[14], D[29], fma(Lbar[13], D[28], fma(Lbar[12], D[27], fma(Lbar[11], D[25], fma(Lbar[10], D[24], fma(Lbar[9], D[22], fma(Lbar[8], D[19], fma(Lbar[7], D[18], fma(Lbar[6], D[17], fma(Lbar[5], D[15], fma(Lbar[4], D[14], fma(Lbar[3], D[12], fma(Lbar[2], D[9], fma(Lbar[1], D[8], Lbar[0] * D[6])))))))))))))))))), nu[3]);
  nu[4] = fma(T(0.5), fma(Lbar[8], D[25], fma(Lbar[7], D[24], fma(Lbar[6], D[23], fma(Lbar[5], D[22], fma(Lbar[4], D[21], fma(Lbar[3], D[20], fma(Lbar[2], D[12], fma(Lbar[1], D[11], Lbar[0] * D[10])))))))), nu[4]);
  nu[5] = fma(T(1), fma(Lbar[8], D[28], fma(Lbar[7], D[27], fma(Lbar[6], D[26], fma(Lbar[5], D[24], fma(Lbar[4], D[23], fma(Lbar[3], D[21], fma(Lbar[2], D[14], fma(Lbar[1], D[13], Lbar[0] * D[11])))))))), nu[5]);
  nu[6] = fma(T(1), fma(Lbar[8], D[29], fma(Lbar[7], D[28], fma(Lbar[6], D[27], fma(Lbar[5], D[25], fma(Lbar[4], D[24], fma(Lbar[3], D[22], fma(Lbar[2], D[15], fma(Lbar[1], D[14], Lbar[0] * D[12])))))))), nu[6]);
  nu[7] = fma(T(0.5), fma(Lbar[8], D[32], fma(Lbar[7], D[31], fma(Lbar[6], D[30], fma(Lbar[5], D[27], fma(Lbar[4], D[26], fma(Lbar[3], D[23], fma(Lbar[2], D[17], fma(Lbar[1], D[16], Lbar[0] * D[13])))))))), nu[7]);
  nu[8] = fma(T(1), fma(Lbar[8], D[33], fma(Lbar[7], D[32], fma(Lbar[6], D[31], fma(Lbar[5], D[28], fma(Lbar[4], D[27], fma(Lbar[3], D[24], fma(Lbar[2], D[18], fma(Lbar[1], D[17], Lbar[0] * D[14])))))))), nu[8]);
  nu[9] = fma(T(0.5), fma(Lbar[8], D[34], fma(Lbar[7], D[33], fma(Lbar[6], D[32], fma(Lbar[5], D[29], fma(Lbar[4], D[28], fma(Lbar[3], D[25], fma(Lbar[2], D[19], fma(Lbar[1], D[18], Lbar[0] * D[15])))))))), nu[9]);
  nu[10] = fma(T(-0.16666666666666666), fma(Lbar[2], D[22], fma(Lbar[1], D[21], Lbar[0] * D[20])), nu[10]);
  nu[11] = fma(T(-0.5), fma(Lbar[2], D[24], fma(Lbar[1], D[23], Lbar[0] * D[21])), nu[11]);
  nu[12] = fma(T(-0.5), fma(Lbar[2], D[25], fma(Lbar[1], D[24], Lbar[0] * D[22])), nu[12]);
  nu[13] = fma(T(-0.5), fma(Lbar[2], D[27], fma(Lbar[1], D[26], Lbar[0] * D[23])), nu[13]);
  nu[14] = fma(T(-1), fma(Lbar[2], D[28], fma(Lbar[1], D[27], Lbar[0] * D[24])), nu[14]);
  nu[15] = fma(T(-0.5), fma(Lbar[2], D[29], fma(Lbar[1], D[28], Lbar[0] * D[25])), nu[15]);
  nu[16] = fma(T(-0.16666666666666666), fma(Lbar[2], D[31], fma(Lbar[1], D[30], Lbar[0] * D[26])), nu[16]);
  nu[17] = fma(T(-0.5), fma(Lbar[2], D[32], fma(Lbar[1], D[31], Lbar[0] * D[27])), nu[17]);
  nu[18] = fma(T(-0.5), fma(Lbar[2], D[33], fma(Lbar[1], D[32], Lbar[0] * D[28])), nu[18]);
  nu[19] = fma(T(-0.16666666666666666), fma(Lbar[2], D[34], fma(Lbar[1], D[33], Lbar[0] * D[29])), nu[19]);
}

template <typename T>
__device__ __forceinline__ void l2p_hess_pe4(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {
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
  ox = fma(-lz * q19, Lc[48], fma(-lz * q18, Lc[47], fma(-lz * q17, Lc[46], fma(-lz * q16, Lc[45], fma(-lz * q15, Lc[43], fma(-lz * q14, Lc[42], fma(-lz * q13, Lc[41], fma(-lz * q12, Lc[39], fma(-lz * q11, Lc[38], fma(-lz * q10, Lc[36], fma(-lz * q9, Lc[28], fma(-lz * q8, Lc[27], fma(-lz * q7, Lc[26], fma(-lz * q6, Lc[24], fma(-lz * q5, Lc[23], fma(-lz * q4, Lc[21], fma(-lz * q3, Lc[14], fma(-lz * q2, Lc[13], fma(-lz * q1, Lc[11], fma(-lz * q0, Lc[5], fma(-ly * q19, Lc[47], fma(-ly * q18, Lc[46], fma(-ly * q17, Lc[45], fma(-ly * q16, Lc[44], fma(-ly * q15, Lc[42], fma(-ly * q14, Lc[41], fma(-ly * q13, Lc[40], fma(-ly * q12, Lc[38], fma(-ly * q11, Lc[37], fma(-ly * q10, Lc[35], fma(-ly * q9, Lc[27], fma(-ly * q8, Lc[26], fma(-ly * q7, Lc[25], fma(-ly * q6, Lc[23], fma(-ly * q5, Lc[22], fma(-ly * q4, Lc[20], fma(-ly * q3, Lc[13], fma(-ly * q2, Lc[12], fma(-ly * q1, Lc[10], fma(-ly * q0, Lc[4], fma(-lx * q19, Lc[43], fma(-lx * q18, Lc[42], fma(-lx * q17, Lc[41], fma(-lx * q16, Lc[40], fma(-lx * q15, Lc[39], fma(-lx * q14, Lc[38], fma(-lx * q13, Lc[37], fma(-lx * q12, Lc[36], fma(-lx * q11, Lc[35], fma(-lx * q10, Lc[34], fma(-lx * q9, Lc[24], fma(-lx * q8, Lc[23], fma(-lx * q7, Lc[22], fma(-lx * q6, Lc[21], fma(-lx * q5, Lc[20], fma(-lx * q4, Lc[19], fma(-lx * q3, Lc[11], fma(-lx * q2, Lc[10], fma(-lx * q1, Lc[9], fma(-lx * q0, Lc[3], ox))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  oy = fma(-lz * q19, Lc[53], fma(-lz * q18, Lc[52], fma(-lz * q17, Lc[51], fma(-lz * q16, Lc[50], fma(-lz * q15, Lc[47], fma(-lz * q14, Lc[46], fma(-lz * q13, Lc[45], fma(-lz * q12, Lc[42], fma(-lz * q11, Lc[41], fma(-lz * q10, Lc[38], fma(-lz * q9, Lc[32], fma(-lz * q8, Lc[31], fma(-lz * q7, Lc[30], fma(-lz * q6, Lc[27], fma(-lz * q5, Lc[26], fma(-lz * q4, Lc[23], fma(-lz * q3, Lc[17], fma(-lz * q2, Lc[16], fma(-lz * q1, Lc[13], fma(-lz * q0, Lc[7], fma(-ly * q19, Lc[52], fma(-ly * q18, Lc[51], fma(-ly * q17, Lc[50], fma(-ly * q16, Lc[49], fma(-ly * q15, Lc[46], fma(-ly * q14, Lc[45], fma(-ly * q13, Lc[44], fma(-ly * q12, Lc[41], fma(-ly * q11, Lc[40], fma(-ly * q10, Lc[37], fma(-ly * q9, Lc[31], fma(-ly * q8, Lc[30], fma(-ly * q7, Lc[29], fma(-ly * q6, Lc[26], fma(-ly * q5, Lc[25], fma(-ly * q4, Lc[22], fma(-ly * q3, Lc[16], fma(-ly * q2, Lc[15], fma(-ly * q1, Lc[12], fma(-ly * q0, Lc[6], fma(-lx * q19, Lc[47], fma(-lx * q18, Lc[46], fma(-lx * q17, Lc[45], fma(-lx * q16, Lc[44], fma(-lx * q15, Lc[42], fma(-lx * q14, Lc[41], fma(-lx * q13, Lc[40], fma(-lx * q12, Lc[38], fma(-lx * q11, Lc[37], fma(-lx * q10, Lc[35], fma(-lx * q9, Lc[27], fma(-lx * q8, Lc[26], fma(-lx * q7, Lc[25], fma(-lx * q6, Lc[23], fma(-lx * q5, Lc[22], fma(-lx * q4, Lc[20], fma(-lx * q3, Lc[13], fma(-lx * q2, Lc[12], fma(-lx * q1, Lc[10], fma(-lx * q0, Lc[4], oy))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  oz = fma(-lz * q19, Lc[54], fma(-lz * q18, Lc[53], fma(-lz * q17, Lc[52], fma(-lz * q16, Lc[51], fma(-lz * q15, Lc[48], fma(-lz * q14, Lc[47], fma(-lz * q13, Lc[46], fma(-lz * q12, Lc[43], fma(-lz * q11, Lc[42], fma(-lz * q10, Lc[39], fma(-lz * q9, Lc[33], fma(-lz * q8, Lc[32], fma(-lz * q7, Lc[31], fma(-lz * q6, Lc[28], fma(-lz * q5, Lc[27], fma(-lz * q4, Lc[24], fma(-lz * q3, Lc[18], fma(-lz * q2, Lc[17], fma(-lz * q1, Lc[14], fma(-lz * q0, Lc[8], fma(-ly * q19, Lc[53], fma(-ly * q18, Lc[52], fma(-ly * q17, Lc[51], fma(-ly * q16, Lc[50], fma(-ly * q15, Lc[47], fma(-ly * q14, Lc[46], fma(-ly * q13, Lc[45], fma(-ly * q12, Lc[42], fma(-ly * q11, Lc[41], fma(-ly * q10, Lc[38], fma(-ly * q9, Lc[32], fma(-ly * q8, Lc[31], fma(-ly * q7, Lc[30], fma(-ly * q6, Lc[27], fma(-ly * q5, Lc[26], fma(-ly * q4, Lc[23], fma(-ly * q3, Lc[17], fma(-ly * q2, Lc[16], fma(-ly * q1, Lc[13], fma(-ly * q0, Lc[7], fma(-lx * q19, Lc[48], fma(-lx * q18, Lc[47], fma(-lx * q17, Lc[46], fma(-lx * q16, Lc[45], fma(-lx * q15, Lc[43], fma(-lx * q14, Lc[42], fma(-lx * q13, Lc[41], fma(-lx * q12, Lc[39], fma(-lx * q11, Lc[38], fma(-lx * q10, Lc[36], fma(-lx * q9, Lc[28], fma(-lx * q8, Lc[27], fma(-lx * q7, Lc[26], fma(-lx * q6, Lc[24], fma(-lx * q5, Lc[23], fma(-lx * q4, Lc[21], fma(-lx * q3, Lc[14], fma(-lx * q2, Lc[13], fma(-lx * q1, Lc[11], fma(-lx * q0, Lc[5], oz))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ void l2p_adj_pe4(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {
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
  Lbar[0] = fma(-lx, q0, Lbar[0]);
  Lbar[1] = fma(-ly, q0, Lbar[1]);
  Lbar[2] = fma(-lz, q0, Lbar[2]);
  Lbar[3] = fma(-lx, q1, Lbar[3]);
  Lbar[4] = fma(-ly, q1, fma(-lx, q2, Lbar[4]));
  Lbar[5] = fma(-lz, q1, fma(-lx, q3, Lbar[5]));
  Lbar[6] = fma(-ly, q2, Lbar[6]);
  Lbar[7] = fma(-lz, q2, fma(-ly, q3, Lbar[7]));
  Lbar[8] = fma(-lz, q3, Lbar[8]);
  Lbar[9] = fma(-lx, q4, Lbar[9]);
  Lbar[10] = fma(-ly, q4, fma(-lx, q5, Lbar[10]));
  Lbar[11] = fma(-lz, q4, fma(-lx, q6, Lbar[11]));
  Lbar[12] = fma(-ly, q5, fma(-lx, q7, Lbar[12]));
  Lbar[13] = fma(-lz, q5, fma(-ly, q6, fma(-lx, q8, Lbar[13])));
  Lbar[14] = fma(-lz, q6, fma(-lx, q9, Lbar[14]));
  Lbar[15] = fma(-ly, q7, Lbar[15]);
  Lbar[16] = fma(-lz, q7, fma(-ly, q8, Lbar[16]));
  Lbar[17] = fma(-lz, q8, fma(-ly, q9, Lbar[17]));
  Lbar[18] = fma(-lz, q9, Lbar[18]);
  Lbar[19] = fma(-lx, q10, Lbar[19]);
  Lbar[20] = fma(-ly, q10, fma(-lx, q11, Lbar[20]));
  Lbar[21] = fma(-lz, q10, fma(-lx, q12, Lbar[21]));
  Lbar[22] = fma(-ly, q11, fma(-lx, q13, Lbar[22]));
  Lbar[23] = fma(-lz, q11, fma(-ly, q12, fma(-lx, q14, Lbar[23])));
  Lbar[24] = fma(-lz, q12, fma(-lx, q15, Lbar[24]));
  Lbar[25] = fma(-ly, q13, fma(-lx, q16, Lbar[25]));
  Lbar[26] = fma(-lz, q13, fma(-ly, q14, fma(-lx, q17, Lbar[26])));
  Lbar[27] = fma(-lz, q14, fma(-ly, q15, fma(-lx, q18, Lbar[27])));
  Lbar[28] = fma(-lz, q15, fma(-lx, q19, Lbar[28]));
  Lbar[29] = fma(-ly, q16, Lbar[29]);
  Lbar[30] = fma(-lz, q16, fma(-ly, q17, Lbar[30]));
  Lbar[31] = fma(-lz, q17, fma(-ly, q18, Lbar[31]));
  Lbar[32] = fma(-lz, q18, fma(-ly, q19, Lbar[32]));
  Lbar[33] = fma(-lz, q19, Lbar[33]);
  Lbar[34] = fma(-lx, q20, Lbar[34]);
  Lbar[35] = fma(-ly, q20, fma(-lx, q21, Lbar[35]));
  Lbar[36] = fma(-lz, q20, fma(-lx, q22, Lbar[36]));
  Lbar[37] = fma(-ly, q21, fma(-lx, q23, Lbar[37]));
  Lbar[38] = fma(-lz, q21, fma(-ly, q22, fma(-lx, q24, Lbar[38])));
  Lbar[39] = fma(-lz, q22, fma(-lx, q25, Lbar[39]));
  Lbar[40] = fma(-ly, q23, fma(-lx, q26, Lbar[40]));
  Lbar[41] = fma(-lz, q23, fma(-ly, q24, fma(-lx, q27, Lbar[41])));
  Lbar[42] = fma(-lz, q24, fma(-ly, q25, fma(-lx, q28, Lbar[42])));
  Lbar[43] = fma(-lz, q25, fma(-lx, q29, Lbar[43]));
  Lbar[44] = fma(-ly, q26, fma(-lx, q30, Lbar[44]));
  Lbar[45] = fma(-lz, q26, fma(-ly, q27, fma(-lx, q31, Lbar[45])));
  Lbar[46] = fma(-lz, q27, fma(-ly, q28, fma(-lx, q32, Lbar[46])));
  Lbar[47] = fma(-lz, q28, fma(-ly, q29, fma(-lx, q33, Lbar[47])));
  Lbar[48] = fma(-lz, q29, fma(-lx, q34, Lbar[48]));
  Lbar[49] = fma(-ly, q30, Lbar[49]);
  Lbar[50] = fma(-lz, q30, fma(-ly, q31, Lbar[50]));
  Lbar[51] = fma(-lz, q31, fma(-ly, q32, Lbar[51]));
  Lbar[52] = fma(-lz, q32, fma(-ly, q33, Lbar[52]));
  Lbar[53] = fma(-lz, q33, fma(-ly, q34, Lbar[53]));
  Lbar[54] = fma(-lz, q34, Lbar[54]);
}
template <typename T>
__device__ __forceinline__ void m2l_adj_pe4(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {
  nu[0] = fma(T(1), fma(Lbar[54], D[55], fma(Lbar[53], D[54], fma(Lbar[52], D[53], fma(Lbar[51], D[52], fma(Lbar[50], D[51], fma(Lbar[49], D[50], fma(Lbar[48], D[49], fma(Lbar[47], D[48], fma(Lbar[46], D[47], fma(Lbar[45], D[46], fma(Lbar[44], D[45], fma(Lbar[43], D[44], fma(Lbar[42], D[43], fma(Lbar[41], D[42], fma(Lbar[40], D[41], fma(Lbar[39], D[40], fma(Lbar[38], D[39], fma(Lbar[37], D[38], fma(Lbar[36], D[37], fma(Lbar[35], D[36], fma(Lbar[34], D[35], fma(Lbar[33], D[34], fma(Lbar[32], D[33], fma(Lbar[31], D[32], fma(Lbar[30], D[31], fma(Lbar[29], D[30], fma(Lbar[28], D[29], fma(Lbar[27], D[28], fma(Lbar[26], D[27], fma(Lbar[25], D[26], fma(Lbar[24], D[25], fma(Lbar[23], D[24], fma(Lbar[22], D[23], fma(Lbar[21], D[22], fma(Lbar[20], D[21], fma(Lbar[19], D[20], fma(Lbar[18], D[19], fma(Lbar[17], D[18], fma(Lbar[16], D[17], fma(Lbar[15], D[16], fma(Lbar[14], D[15], fma(Lbar[13], D[14], fma(Lbar[12], D[13], fma(Lbar[11], D[12], fma(Lbar[10], D[11], fma(Lbar[9], D[10], fma(Lbar[8], D[9], fma(Lbar[7], D[8], fma(Lbar[6], D[7], fma(Lbar[5], D[6], fma(Lbar[4], D[5], fma(Lbar[3], D[4], fma(Lbar[2], D[3], fma(Lbar[1], D[2], Lbar[0] * D[1])))))))))))))))))))))))))))))))))))))))))))))))))))))), nu[0]);
  nu[1] = fma(T(-1), fma(Lbar[33], D[49], fma(Lbar[32], D[48], fma(Lbar[31], D[47], fma(Lbar[30], D[46], fma(Lbar[29], D[45], fma(Lbar[28], D[44], fma(Lbar[27], D[43], fma(Lbar[26], D[42], fma(Lbar[25], D[41], fma(Lbar[24], D[40], fma(Lbar[23], D[39], fma(Lbar[22], D[38], fma(Lbar[21], D[37], fma(Lbar[20], D[36], fma(Lbar[19], D[35], fma(Lbar[18], D[29], fma(Lbar[17], D[28], fma(Lbar[16], D[27], fma(Lbar[15], D[26], fma(Lbar[14], D[25], fma(Lbar[13], D[24], fma(Lbar[12], D[23], fma(Lbar[11], D[22], fma(Lbar[10], D[21], fma(Lbar[9], D[20], fma(Lbar[8], D[15], fma(Lbar[7], D[14], fma(Lbar[6], D[13], fma(Lbar[5], D[12], fma(Lbar[4], D[11], fma(Lbar[3], D[10], fma(Lbar[2], D[6], fma(Lbar[1], D[5], Lbar[0] * D[4]))))))))))))))))))))))))))))))))), nu[1]);
  nu[2] = fma(T(-1), fma(Lbar[33], D[54], fma(Lbar[32], D[53], fma(Lbar[31], D[52], fma(Lbar[30], D[51], fma(Lbar[29], D[50], fma(Lbar[28], D[48], fma(Lbar[27], D[47], fma(Lbar[26], D[46], fma(Lbar[25], D[45], fma(Lbar[24], D[43], fma(Lbar[23], D[42], fma(Lbar[22], D[41], fma(Lbar[21], D[39], fma(Lbar[20], D[38], fma(Lbar[19], D[36], fma(Lbar[18], D[33], fma(Lbar[17], D[32], fma(Lbar[16], D[31], fma(Lbar[15], D[30], fma(Lbar[14], D[28], fma(Lbar[13], D[27], fma(Lbar[12], D[26], fma(Lbar[11], D[24], fma(Lbar[10], D[23], fma(Lbar[9], D[21], fma(Lbar[8], D[18], fma(Lbar[7], D[17], fma(Lbar[6], D[16], fma(Lbar[5], D[14], fma(Lbar[4], D[13], fma(Lbar[3], D[11], fma(Lbar[2], D[8], fma(Lbar[1], D[7], Lbar[0] * D[5]))))))))))))))))))))))))))))))))), nu[2]);
  nu[3] = fma(T(-1), fma(Lbar[33], D[55], fma(Lbar[32], D[54], fma(Lbar[31], D[53], fma(Lbar[30], D[52], fma(Lbar[29], D[51], fma(Lbar[28], D[49], fma(Lbar[27], D[48], fma(Lbar[26], D[47], fma(Lbar[25], D[46], fma(Lbar[24], D[44], fma(Lbar[23], D[43], fma(Lbar[22], D[42], fma(Lbar[21], D[40], fma(Lbar[20], D[39], fma(Lbar[19], D[37], fma(Lbar[18], D[34], fma(Lbar[17], D[33], fma(Lbar[16], D[32], fma(Lbar[15], D[31], fma(Lbar[14], D[29], fma(Lbar[13], D[28], fma(Lbar[12], D[27], fma(Lbar[11], D[25], fma(Lbar[10], D[24], fma(Lbar[9], D[22], fma(Lbar[8], D[19], fma(Lbar[7], D[18], fma(Lbar[6], D[17], fma(Lbar[5], D[15], fma(Lbar[4], D[14], fma(Lbar[3], D[12], fma(Lbar[2], D[9], fma(Lbar[1], D[8], Lbar[0] * D[6]))))))))))))))))))))))))))))))))), nu[3]);
  nu[4] = fma(T(0.5), fma(Lbar[18], D[44], fma(Lbar[17], D[43], fma(Lbar[16], D[42], fma(Lbar[15], D[41], fma(Lbar[14], D[40], fma(Lbar[13], D[39], fma(Lbar[12], D[38], fma(Lbar[11], D[37], fma(Lbar[10], D[36], fma(Lbar[9], D[35], fma(Lbar[8], D[25], fma(Lbar[7], D[24], fma(Lbar[6], D[23], fma(Lbar[5], D[22], fma(Lbar[4], D[21], fma(Lbar[3], D[20], fma(Lbar[2], D[12], fma(Lbar[1], D[11], Lbar[0] * D[10])))))))))))))))))), nu[4]);
  nu[5] = fma(T(1), fma(Lbar[18], D[48], fma(Lbar[17], D[47], fma(Lbar[16], D[46], fma(Lbar[15], D[45], fma(Lbar[14], D[43], fma(Lbar[13], D[42], fma(Lbar[12], D[41], fma(Lbar[11], D[39], fma(Lbar[10], D[38], fma(Lbar[9], D[36], fma(Lbar[8], D[28], fma(Lbar[7], D[27], fma(Lbar[6], D[26], fma(Lbar[5], D[24], fma(Lbar[4], D[23], fma(Lbar[3], D[21], fma(Lbar[2], D[14], fma(Lbar[1], D[13], Lbar[0] * D[11])))))))))))))))))), nu[5]);
  nu[6] = fma(T(1), fma(Lbar[18], D[49], fma(Lbar[17], D[48], fma(Lbar[16], D[47], fma(Lbar[15], D[46], fma(Lbar[14], D[44], fma(Lbar[13], D[43], fma(Lbar[12], D[42], fma(Lbar[11], D[40], fma(Lbar[10], D[39], fma(Lbar[9], D[37], fma(Lbar[8], D[29], fma(Lbar[7], D[28], fma(Lbar[6], D[27], fma(Lbar[5], D[25], fma(Lbar[4], D[24], fma(Lbar[3], D[22], fma(Lbar[2], D[15], fma(Lbar[1], D[14], Lbar[0] * D[12])))))))))))))))))), nu[6]);
  nu[7] = fma(T(0.5), fma(Lbar[18], D[53], fma(Lbar[17], D[52], fma(Lbar[16], D[51], fma(Lbar[15], D[50], fma(Lbar[14], D[47], fma(Lbar[13], D[46], fma(Lbar[12], D[45], fma(Lbar[11], D[42], fma(Lbar[10], D[41], fma(Lbar[9], D[38], fma(Lbar[8], D[32], fma(Lbar[7], D[31], fma(Lbar[6], D[30], fma(Lbar[5], D[27], fma(Lbar[4], D[26], fma(Lbar[3], D[23], fma(Lbar[2], D[17], fma(Lbar[1], D[16], Lbar[0] * D[13])))))))))))))))))), nu[7]);
  nu[8] = fma(T(1), fma(Lbar[18], D[54], fma(Lbar[17], D[53], fma(Lbar[16], D[52], fma(Lbar[15], D[51], fma(Lbar[14], D[48], fma(Lbar[13], D[47], fma(Lbar[12], D[46], fma(Lbar[11], D[43], fma(Lbar[10], D[42], fma(Lbar[9], D[39], fma(Lbar[8], D[33], fma(Lbar[7], D[32], fma(Lbar[6], D[31], fma(Lbar[5], D[28], fma(Lbar[4], D[27], fma(Lbar[3], D[24], fma(Lbar[2], D[18], fma(Lbar[1], D[17], Lbar[0] * D[14])))))))))))))))))), nu[8]);
  nu[9] = fma(T(0.5), fma(Lbar[18], D[55], fma(Lbar[17], D[54], fma(Lbar[16], D[53], fma(Lbar[15], D[52], fma(Lbar[14], D[49], fma(Lbar[13], D[48], fma(Lbar[12], D[47], fma(Lbar[11], D[44], fma(Lbar[10], D[43], fma(Lbar[9], D[40], fma(Lbar[8], D[34], fma(Lbar[7], D[33], fma(Lbar[6], D[32], fma(Lbar[5], D[29], fma(Lbar[4], D[28], fma(Lbar[3], D[25], fma(Lbar[2], D[19], fma(Lbar[1], D[18], Lbar[0] * D[15])))))))))))))))))), nu[9]);
  nu[10] = fma(T(-0.16666666666666666), fma(Lbar[8], D[40], fma(Lbar[7], D[39], fma(Lbar[6], D[38], fma(Lbar[5], D[37], fma(Lbar[4], D[36], fma(Lbar[3], D[35], fma(Lbar[2], D[22], fma(Lbar[1], D[21], Lbar[0] * D[20])))))))), nu[10]);
  nu[11] = fma(T(-0.5), fma(Lbar[8], D[43], fma(Lbar[7], D[42], fma(Lbar[6], D[41], fma(Lbar[5], D[39], fma(Lbar[4], D[38], fma(Lbar[3], D[36], fma(Lbar[2], D[24], fma(Lbar[1], D[23], Lbar[0] * D[21])))))))), nu[11]);
  nu[12] = fma(T(-0.5), fma(Lbar[8], D[44], fma(Lbar[7], D[43], fma(Lbar[6], D[42], fma(Lbar[5], D[40], fma(Lbar[4], D[39], fma(Lbar[3], D[37], fma(Lbar[2], D[25], fma(Lbar[1], D[24], Lbar[0] * D[22])))))))), nu[12]);
  nu[13] = fma(T(-0.5), fma(Lbar[8], D[47], fma(Lbar[7], D[46], fma(Lbar[6], D[45], fma(Lbar[5], D[42], fma(Lbar[4], D[41], fma(Lbar[3], D[38], fma(Lbar[2], D[27], fma(Lbar[1], D[26], Lbar[0] * D[23])))))))), nu[13]);
  nu[14] = fma(T(-1), fma(Lbar[8], D[48], fma(Lbar[7], D[47], fma(Lbar[6], D[46], fma(Lbar[5], D[43], fma(Lbar[4], D[42], fma(Lbar[3], D[39], fma(Lbar[2], D[28], fma(Lbar[1], D[27], Lbar[0] * D[24])))))))), nu[14]);
  nu[15] = fma(T(-0.5), fma(Lbar[8], D[49], fma(Lbar[7], D[48], fma(Lbar[6], D[47], fma(Lbar[5], D[44], fma(Lbar[4], D[43], fma(Lbar[3], D[40], fma(Lbar[2], D[29], fma(Lbar[1], D[28], Lbar[0] * D[25])))))))), nu[15]);
  nu[16] = fma(T(-0.16666666666666666), fma(Lbar[8], D[52], fma(Lbar[7], D[51], fma(Lbar[6], D[50], fma(Lbar[5], D[46], fma(Lbar[4], D[45], fma(Lbar[3], D[41], fma(Lbar[2], D[31], fma(Lbar[1], D[30], Lbar[0] * D[26])))))))), nu[16]);
  nu[17] = fma(T(-0.5), fma(Lbar[8], D[53], fma(Lbar[7], D[52], fma(Lbar[6], D[51], fma(Lbar[5], D[47], fma(Lbar[4], D[46], fma(Lbar[3], D[42], fma(Lbar[2], D[32], fma(Lbar[1], D[31], Lbar[0] * D[27])))))))), nu[17]);
  nu[18] = fma(T(-0.5), fma(Lbar[8], D[54], fma(Lbar[7], D[53], fma(Lbar[6], D[52], fma(Lbar[5], D[48], fma(Lbar[4], D[47], fma(Lbar[3], D[43], fma(Lbar[2], D[33], fma(Lbar[1], D[32], Lbar[0] * D[28])))))))), nu[18]);
  nu[19] = fma(T(-0.16666666666666666), fma(Lbar[8], D[55], fma(Lbar[7], D[54], fma(Lbar[6], D[53], fma(Lbar[5], D[49], fma(Lbar[4], D[48], fma(Lbar[3], D[44], fma(Lbar[2], D[34], fma(Lbar[1], D[33], Lbar[0] * D[29])))))))), nu[19]);
  nu[20] = fma(T(0.041666666666666664), fma(Lbar[2], D[37], fma(Lbar[1], D[36], Lbar[0] * D[35])), nu[20]);
  nu[21] = fma(T(0.16666666666666666), fma(Lbar[2], D[39], fma(Lbar[1], D[38], Lbar[0] * D[36])), nu[21]);
  nu[22] = fma(T(0.16666666666666666), fma(Lbar[2], D[40], fma(Lbar[1], D[39], Lbar[0] * D[37])), nu[22]);
  nu[23] = fma(T(0.25), fma(Lbar[2], D[42], fma(Lbar[1], D[41], Lbar[0] * D[38])), nu[23]);
  nu[24] = fma(T(0.5), fma(Lbar[2], D[43], fma(Lbar[1], D[42], Lbar[0] * D[39])), nu[24]);
  nu[25] = fma(T(0.25), fma(Lbar[2], D[44], fma(Lbar[1], D[43], Lbar[0] * D[40])), nu[25]);
  nu[26] = fma(T(0.16666666666666666), fma(Lbar[2], D[46], fma(Lbar[1], D[45], Lbar[0] * D[41])), nu[26]);
  nu[27] = fma(T(0.5), fma(Lbar[2], D[47], fma(Lbar[1], D[46], Lbar[0] * D[42])), nu[27]);
  nu[28] = fma(T(0.5), fma(Lbar[2], D[48], fma(Lbar[1], D[47], Lbar[0] * D[43])), nu[28]);
  nu[29] = fma(T(0.16666666666666666), fma(Lbar[2], D[49], fma(Lbar[1], D[48], Lbar[0] * D[44])), nu[29]);
  nu[30] = fma(T(0.041666666666666664), fma(Lbar[2], D[51], fma(Lbar[1], D[50], Lbar[0] * D[45])), nu[30]);
  nu[31] = fma(T(0.16666666666666666), fma(Lbar[2], D[52], fma(Lbar[1], D[51], Lbar[0] * D[46])), nu[31]);
  nu[32] = fma(T(0.25), fma(Lbar[2], D[53], fma(Lbar[1], D[52], Lbar[0] * D[47])), nu[32]);
  nu[33] = fma(T(0.16666666666666666), fma(Lbar[2], D[54], fma(Lbar[1], D[53], Lbar[0] * D[48])), nu[33]);
  nu[34] = fma(T(0.041666666666666664), fma(Lbar[2], D[55], fma(Lbar[1], D[54], Lbar[0] * D[49])), nu[34]);
}

template <typename T>
__device__ __forceinline__ void l2p_hess_pe5(const T* __restrict__ Lc, T dx, T dy, T dz, T lx, T ly, T lz, T& ox, T& oy, T& oz) {
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
  ox = fma(-lz * q34, Lc[75], fma(-lz * q33, Lc[74], fma(-lz * q32, Lc[73], fma(-lz * q31, Lc[72], fma(-lz * q30, Lc[71], fma(-lz * q29, Lc[69], fma(-lz * q28, Lc[68], fma(-lz * q27, Lc[67], fma(-lz * q26, Lc[66], fma(-lz * q25, Lc[64], fma(-lz * q24, Lc[63], fma(-lz * q23, Lc[62], fma(-lz * q22, Lc[60], fma(-lz * q21, Lc[59], fma(-lz * q20, Lc[57], fma(-lz * q19, Lc[48], fma(-lz * q18, Lc[47], fma(-lz * q17, Lc[46], fma(-lz * q16, Lc[45], fma(-lz * q15, Lc[43], fma(-lz * q14, Lc[42], fma(-lz * q13, Lc[41], fma(-lz * q12, Lc[39], fma(-lz * q11, Lc[38], fma(-lz * q10, Lc[36], fma(-lz * q9, Lc[28], fma(-lz * q8, Lc[27], fma(-lz * q7, Lc[26], fma(-lz * q6, Lc[24], fma(-lz * q5, Lc[23], fma(-lz * q4, Lc[21], fma(-lz * q3, Lc[14], fma(-lz * q2, Lc[13], fma(-lz * q1, Lc[11], fma(-lz * q0, Lc[5], fma(-ly * q34, Lc[74], fma(-ly * q33, Lc[73], fma(-ly * q32, Lc[72], fma(-ly * q31, Lc[71], fma(-ly * q30, Lc[70], fma(-ly * q29, Lc[68], fma(-ly * q28, Lc[67], fma(-ly * q27, Lc[66], fma(-ly * q26, Lc[65], fma(-ly * q25, Lc[63], fma(-ly * q24, Lc[62], fma(-ly * q23, Lc[61], fma(-ly * q22, Lc[59], fma(-ly * q21, Lc[58], fma(-ly * q20, Lc[56], fma(-ly * q19, Lc[47], fma(-ly * q18, Lc[46], fma(-ly * q17, Lc[45], fma(-ly * q16, Lc[44], fma(-ly * q15, Lc[42], fma(-ly * q14, Lc[41], fma(-ly * q13, Lc[40], fma(-ly * q12, Lc[38], fma(-ly * q11, Lc[37], fma(-ly * q10, Lc[35], fma(-ly * q9, Lc[27], fma(-ly * q8, Lc[26], fma(-ly * q7, Lc[25], fma(-ly * q6, Lc[23], fma(-ly * q5, Lc[22], fma(-ly * q4, Lc[20], fma(-ly * q3, Lc[13], fma(-ly * q2, Lc[12], fma(-ly * q1, Lc[10], fma(-ly * q0, Lc[4], fma(-lx * q34, Lc[69], fma(-lx * q33, Lc[68], fma(-lx * q32, Lc[67], fma(-lx * q31, Lc[66], fma(-lx * q30, Lc[65], fma(-lx * q29, Lc[64], fma(-lx * q28, Lc[63], fma(-lx * q27, Lc[62], fma(-lx * q26, Lc[61], fma(-lx * q25, Lc[60], fma(-lx * q24, Lc[59], fma(-lx * q23, Lc[58], fma(-lx * q22, Lc[57], fma(-lx * q21, Lc[56], fma(-lx * q20, Lc[55], fma(-lx * q19, Lc[43], fma(-lx * q18, Lc[42], fma(-lx * q17, Lc[41], fma(-lx * q16, Lc[40], fma(-lx * q15, Lc[39], fma(-lx * q14, Lc[38], fma(-lx * q13, Lc[37], fma(-lx * q12, Lc[36], fma(-lx * q11, Lc[35], fma(-lx * q10, Lc[34], fma(-lx * q9, Lc[24], fma(-lx * q8, Lc[23], fma(-lx * q7, Lc[22], fma(-lx * q6, Lc[21], fma(-lx * q5, Lc[20], fma(-lx * q4, Lc[19], fma(-lx * q3, Lc[11], fma(-lx * q2, Lc[10], fma(-lx * q1, Lc[9], fma(-lx * q0, Lc[3], ox)))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  oy = fma(-lz * q34, Lc[81], fma(-lz * q33, Lc[80], fma(-lz * q32, Lc[79], fma(-lz * q31, Lc[78], fma(-lz * q30, Lc[77], fma(-lz * q29, Lc[74], fma(-lz * q28, Lc[73], fma(-lz * q27, Lc[72], fma(-lz * q26, Lc[71], fma(-lz * q25, Lc[68], fma(-lz * q24, Lc[67], fma(-lz * q23, Lc[66], fma(-lz * q22, Lc[63], fma(-lz * q21, Lc[62], fma(-lz * q20, Lc[59], fma(-lz * q19, Lc[53], fma(-lz * q18, Lc[52], fma(-lz * q17, Lc[51], fma(-lz * q16, Lc[50], fma(-lz * q15, Lc[47], fma(-lz * q14, Lc[46], fma(-lz * q13, Lc[45], fma(-lz * q12, Lc[42], fma(-lz * q11, Lc[41], fma(-lz * q10, Lc[38], fma(-lz * q9, Lc[32], fma(-lz * q8, Lc[31], fma(-lz * q7, Lc[30], fma(-lz * q6, Lc[27], fma(-lz * q5, Lc[26], fma(-lz * q4, Lc[23], fma(-lz * q3, Lc[17], fma(-lz * q2, Lc[16], fma(-lz * q1, Lc[13], fma(-lz * q0, Lc[7], fma(-ly * q34, Lc[80], fma(-ly * q33, Lc[79], fma(-ly * q32, Lc[78], fma(-ly * q31, Lc[77], fma(-ly * q30, Lc[76], fma(-ly * q29, Lc[73], fma(-ly * q28, Lc[72], fma(-ly * q27, Lc[71], fma(-ly * q26, Lc[70], fma(-ly * q25, Lc[67], fma(-ly * q24, Lc[66], fma(-ly * q23, Lc[65], fma(-ly * q22, Lc[62], fma(-ly * q21, Lc[61], fma(-ly * q20, Lc[58], fma(-ly * q19, Lc[52], fma(-ly * q18, Lc[51], fma(-ly * q17, Lc[50], fma(-ly * q16, Lc[49], fma(-ly * q15, Lc[46], fma(-ly * q14, Lc[45], fma(-ly * q13, Lc[44], fma(-ly * q12, Lc[41], fma(-ly * q11, Lc[40], fma(-ly * q10, Lc[37], fma(-ly * q9, Lc[31], fma(-ly * q8, Lc[30], fma(-ly * q7, Lc[29], fma(-ly * q6, Lc[26], fma(-ly * q5, Lc[25], fma(-ly * q4, Lc[22], fma(-ly * q3, Lc[16], fma(-ly * q2, Lc[15], fma(-ly * q1, Lc[12], fma(-ly * q0, Lc[6], fma(-lx * q34, Lc[74], fma(-lx * q33, Lc[73], fma(-lx * q32, Lc[72], fma(-lx * q31, Lc[71], fma(-lx * q30, Lc[70], fma(-lx * q29, Lc[68], fma(-lx * q28, Lc[67], fma(-lx * q27, Lc[66], fma(-lx * q26, Lc[65], fma(-lx * q25, Lc[63], fma(-lx * q24, Lc[62], fma(-lx * q23, Lc[61], fma(-lx * q22, Lc[59], fma(-lx * q21, Lc[58], fma(-lx * q20, Lc[56], fma(-lx * q19, Lc[47], fma(-lx * q18, Lc[46], fma(-lx * q17, Lc[45], fma(-lx * q16, Lc[44], fma(-lx * q15, Lc[42], fma(-lx * q14, Lc[41], fma(-lx * q13, Lc[40], fma(-lx * q12, Lc[38], fma(-lx * q11, Lc[37], fma(-lx * q10, Lc[35], fma(-lx * q9, Lc[27], fma(-lx * q8, Lc[26], fma(-lx * q7, Lc[25], fma(-lx * q6, Lc[23], fma(-lx * q5, Lc[22], fma(-lx * q4, Lc[20], fma(-lx * q3, Lc[13], fma(-lx * q2, Lc[12], fma(-lx * q1, Lc[10], fma(-lx * q0, Lc[4], oy)))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
  oz = fma(-lz * q34, Lc[82], fma(-lz * q33, Lc[81], fma(-lz * q32, Lc[80], fma(-lz * q31, Lc[79], fma(-lz * q30, Lc[78], fma(-lz * q29, Lc[75], fma(-lz * q28, Lc[74], fma(-lz * q27, Lc[73], fma(-lz * q26, Lc[72], fma(-lz * q25, Lc[69], fma(-lz * q24, Lc[68], fma(-lz * q23, Lc[67], fma(-lz * q22, Lc[64], fma(-lz * q21, Lc[63], fma(-lz * q20, Lc[60], fma(-lz * q19, Lc[54], fma(-lz * q18, Lc[53], fma(-lz * q17, Lc[52], fma(-lz * q16, Lc[51], fma(-lz * q15, Lc[48], fma(-lz * q14, Lc[47], fma(-lz * q13, Lc[46], fma(-lz * q12, Lc[43], fma(-lz * q11, Lc[42], fma(-lz * q10, Lc[39], fma(-lz * q9, Lc[33], fma(-lz * q8, Lc[32], fma(-lz * q7, Lc[31], fma(-lz * q6, Lc[28], fma(-lz * q5, Lc[27], fma(-lz * q4, Lc[24], fma(-lz * q3, Lc[18], fma(-lz * q2, Lc[17], fma(-lz * q1, Lc[14], fma(-lz * q0, Lc[8], fma(-ly * q34, Lc[81], fma(-ly * q33, Lc[80], fma(-ly * q32, Lc[79], fma(-ly * q31, Lc[78], fma(-ly * q30, Lc[77], fma(-ly * q29, Lc[74], fma(-ly * q28, Lc[73], fma(-ly * q27, Lc[72], fma(-ly * q26, Lc[71], fma(-ly * q25, Lc[68], fma(-ly * q24, Lc[67], fma(-ly * q23, Lc[66], fma(-ly * q22, Lc[63], fma(-ly * q21, Lc[62], fma(-ly * q20, Lc[59], fma(-ly * q19, Lc[53], fma(-ly * q18, Lc[52], fma(-ly * q17, Lc[51], fma(-ly * q16, Lc[50], fma(-ly * q15, Lc[47], fma(-ly * q14, Lc[46], fma(-ly * q13, Lc[45], fma(-ly * q12, Lc[42], fma(-ly * q11, Lc[41], fma(-ly * q10, Lc[38], fma(-ly * q9, Lc[32], fma(-ly * q8, Lc[31], fma(-ly * q7, Lc[30], fma(-ly * q6, Lc[27], fma(-ly * q5, Lc[26], fma(-ly * q4, Lc[23], fma(-ly * q3, Lc[17], fma(-ly * q2, Lc[16], fma(-ly * q1, Lc[13], fma(-ly * q0, Lc[7], fma(-lx * q34, Lc[75], fma(-lx * q33, Lc[74], fma(-lx * q32, Lc[73], fma(-lx * q31, Lc[72], fma(-lx * q30, Lc[71], fma(-lx * q29, Lc[69], fma(-lx * q28, Lc[68], fma(-lx * q27, Lc[67], fma(-lx * q26, Lc[66], fma(-lx * q25, Lc[64], fma(-lx * q24, Lc[63], fma(-lx * q23, Lc[62], fma(-lx * q22, Lc[60], fma(-lx * q21, Lc[59], fma(-lx * q20, Lc[57], fma(-lx * q19, Lc[48], fma(-lx * q18, Lc[47], fma(-lx * q17, Lc[46], fma(-lx * q16, Lc[45], fma(-lx * q15, Lc[43], fma(-lx * q14, Lc[42], fma(-lx * q13, Lc[41], fma(-lx * q12, Lc[39], fma(-lx * q11, Lc[38], fma(-lx * q10, Lc[36], fma(-lx * q9, Lc[28], fma(-lx * q8, Lc[27], fma(-lx * q7, Lc[26], fma(-lx * q6, Lc[24], fma(-lx * q5, Lc[23], fma(-lx * q4, Lc[21], fma(-lx * q3, Lc[14], fma(-lx * q2, Lc[13], fma(-lx * q1, Lc[11], fma(-lx * q0, Lc[5], oz)))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))));
}
template <typename T>
__device__ __forceinline__ void l2p_adj_pe5(T dx, T dy, T dz, T lx, T ly, T lz, T* __restrict__ Lbar) {
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
  Lbar[0] = fma(-lx, q0, Lbar[0]);
  Lbar[1] = fma(-ly, q0, Lbar[1]);
  Lbar[2] = fma(-lz, q0, Lbar[2]);
  Lbar[3] = fma(-lx, q1, Lbar[3]);
  Lbar[4] = fma(-ly, q1, fma(-lx, q2, Lbar[4]));
  Lbar[5] = fma(-lz, q1, fma(-lx, q3, Lbar[5]));
  Lbar[6] = fma(-ly, q2, Lbar[6]);
  Lbar[7] = fma(-lz, q2, fma(-ly, q3, Lbar[7]));
  Lbar[8] = fma(-lz, q3, Lbar[8]);
  Lbar[9] = fma(-lx, q4, Lbar[9]);
  Lbar[10] = fma(-ly, q4, fma(-lx, q5, Lbar[10]));
  Lbar[11] = fma(-lz, q4, fma(-lx, q6, Lbar[11]));
  Lbar[12] = fma(-ly, q5, fma(-lx, q7, Lbar[12]));
  Lbar[13] = fma(-lz, q5, fma(-ly, q6, fma(-lx, q8, Lbar[13])));
  Lbar[14] = fma(-lz, q6, fma(-lx, q9, Lbar[14]));
  Lbar[15] = fma(-ly, q7, Lbar[15]);
  Lbar[16] = fma(-lz, q7, fma(-ly, q8, Lbar[16]));
  Lbar[17] = fma(-lz, q8, fma(-ly, q9, Lbar[17]));
  Lbar[18] = fma(-lz, q9, Lbar[18]);
  Lbar[19] = fma(-lx, q10, Lbar[19]);
  Lbar[20] = fma(-ly, q10, fma(-lx, q11, Lbar[20]));
  Lbar[21] = fma(-lz, q10, fma(-lx, q12, Lbar[21]));
  Lbar[22] = fma(-ly, q11, fma(-lx, q13, Lbar[22]));
  Lbar[23] = fma(-lz, q11, fma(-ly, q12, fma(-lx, q14, Lbar[23])));
  Lbar[24] = fma(-lz, q12, fma(-lx, q15, Lbar[24]));
  Lbar[25] = fma(-ly, q13, fma(-lx, q16, Lbar[25]));
  Lbar[26] = fma(-lz, q13, fma(-ly, q14, fma(-lx, q17, Lbar[26])));
  Lbar[27] = fma(-lz, q14, fma(-ly, q15, fma(-lx, q18, Lbar[27])));
  Lbar[28] = fma(-lz, q15, fma(-lx, q19, Lbar[28]));
  Lbar[29] = fma(-ly, q16, Lbar[29]);
  Lbar[30] = fma(-lz, q16, fma(-ly, q17, Lbar[30]));
  Lbar[31] = fma(-lz, q17, fma(-ly, q18, Lbar[31]));
  Lbar[32] = fma(-lz, q18, fma(-ly, q19, Lbar[32]));
  Lbar[33] = fma(-lz, q19, Lbar[33]);
  Lbar[34] = fma(-lx, q20, Lbar[34]);
  Lbar[35] = fma(-ly, q20, fma(-lx, q21, Lbar[35]));
  Lbar[36] = fma(-lz, q20, fma(-lx, q22, Lbar[36]));
  Lbar[37] = fma(-ly, q21, fma(-lx, q23, Lbar[37]));
  Lbar[38] = fma(-lz, q21, fma(-ly, q22, fma(-lx, q24, Lbar[38])));
  Lbar[39] = fma(-lz, q22, fma(-lx, q25, Lbar[39]));
  Lbar[40] = fma(-ly, q23, fma(-lx, q26, Lbar[40]));
  Lbar[41] = fma(-lz, q23, fma(-ly, q24, fma(-lx, q27, Lbar[41])));
  Lbar[42] = fma(-lz, q24, fma(-ly, q25, fma(-lx, q28, Lbar[42])));
  Lbar[43] = fma(-lz, q25, fma(-lx, q29, Lbar[43]));
  Lbar[44] = fma(-ly, q26, fma(-lx, q30, Lbar[44]));
  Lbar[45] = fma(-lz, q26, fma(-ly, q27, fma(-lx, q31, Lbar[45])));
  Lbar[46] = fma(-lz, q27, fma(-ly, q28, fma(-lx, q32, Lbar[46])));
  Lbar[47] = fma(-lz, q28, fma(-ly, q29, fma(-lx, q33, Lbar[47])));
  Lbar[48] = fma(-lz, q29, fma(-lx, q34, Lbar[48]));
  Lbar[49] = fma(-ly, q30, Lbar[49]);
  Lbar[50] = fma(-lz, q30, fma(-ly, q31, Lbar[50]));
  Lbar[51] = fma(-lz, q31, fma(-ly, q32, Lbar[51]));
  Lbar[52] = fma(-lz, q32, fma(-ly, q33, Lbar[52]));
  Lbar[53] = fma(-lz, q33, fma(-ly, q34, Lbar[53]));
  Lbar[54] = fma(-lz, q34, Lbar[54]);
  Lbar[55] = fma(-lx, q35, Lbar[55]);
  Lbar[56] = fma(-ly, q35, fma(-lx, q36, Lbar[56]));
  Lbar[57] = fma(-lz, q35, fma(-lx, q37, Lbar[57]));
  Lbar[58] = fma(-ly, q36, fma(-lx, q38, Lbar[58]));
  Lbar[59] = fma(-lz, q36, fma(-ly, q37, fma(-lx, q39, Lbar[59])));
  Lbar[60] = fma(-lz, q37, fma(-lx, q40, Lbar[60]));
  Lbar[61] = fma(-ly, q38, fma(-lx, q41, Lbar[61]));
  Lbar[62] = fma(-lz, q38, fma(-ly, q39, fma(-lx, q42, Lbar[62])));
  Lbar[63] = fma(-lz, q39, fma(-ly, q40, fma(-lx, q43, Lbar[63])));
  Lbar[64] = fma(-lz, q40, fma(-lx, q44, Lbar[64]));
  Lbar[65] = fma(-ly, q41, fma(-lx, q45, Lbar[65]));
  Lbar[66] = fma(-lz, q41, fma(-ly, q42, fma(-lx, q46, Lbar[66])));
  Lbar[67] = fma(-lz, q42, fma(-ly, q43, fma(-lx, q47, Lbar[67])));
  Lbar[68] = fma(-lz, q43, fma(-ly, q44, fma(-lx, q48, Lbar[68])));
  Lbar[69] = fma(-lz, q44, fma(-lx, q49, Lbar[69]));
  Lbar[70] = fma(-ly, q45, fma(-lx, q50, Lbar[70]));
  Lbar[71] = fma(-lz, q45, fma(-ly, q46, fma(-lx, q51, Lbar[71])));
  Lbar[72] = fma(-lz, q46, fma(-ly, q47, fma(-lx, q52, Lbar[72])));
  Lbar[73] = fma(-lz, q47, fma(-ly, q48, fma(-lx, q53, Lbar[73])));
  Lbar[74] = fma(-lz, q48, fma(-ly, q49, fma(-lx, q54, Lbar[74])));
  Lbar[75] = fma(-lz, q49, fma(-lx, q55, Lbar[75]));
  Lbar[76] = fma(-ly, q50, Lbar[76]);
  Lbar[77] = fma(-lz, q50, fma(-ly, q51, Lbar[77]));
  Lbar[78] = fma(-lz, q51, fma(-ly, q52, Lbar[78]));
  Lbar[79] = fma(-lz, q52, fma(-ly, q53, Lbar[79]));
  Lbar[80] = fma(-lz, q53, fma(-ly, q54, Lbar[80]));
  Lbar[81] = fma(-lz, q54, fma(-ly, q55, Lbar[81]));
  Lbar[82] = fma(-lz, q55, Lbar[82]);
}
template <typename T>
__device__ __forceinline__ void m2l_adj_pe5(const T* __restrict__ Lbar, const T* __restrict__ D, T* __restrict__ nu) {
  nu[0] = fma(T(1), fma(Lbar[82], D[83], fma(Lbar[81], D[82], fma(Lbar[80], D[81], fma(Lbar[79], D[80], fma(Lbar[78], D[79], fma(Lbar[77], D[78], fma(Lbar[76], D[77], fma(Lbar[75], D[76], fma(Lbar[74], D[75], fma(Lbar[73], D[74], fma(Lbar[72], D[73], fma(Lbar[71], D[72], fma(Lbar[70], D[71], fma(Lbar[69], D[70], fma(Lbar[68], D[69], fma(Lbar[67], D[68], fma(Lbar[66], D[67], fma(Lbar[65], D[66], fma(Lbar[64], D[65], fma(Lbar[63], D[64], fma(Lbar[62], D[63], fma(Lbar[61], D[62], fma(Lbar[60], D[61], fma(Lbar[59], D[60], fma(Lbar[58], D[59], fma(Lbar[57], D[58], fma(Lbar[56], D[57], fma(Lbar[55], D[56], fma(Lbar[54], D[55], fma(Lbar[53], D[54], fma(Lbar[52], D[53], fma(Lbar[51], D[52], fma(Lbar[50], D[51], fma(Lbar[49], D[50], fma(Lbar[48], D[49], fma(Lbar[47], D[48], fma(Lbar[46], D[47], fma(Lbar[45], D[46], fma(Lbar[44], D[45], fma(Lbar[43], D[44], fma(Lbar[42], D[43], fma(Lbar[41], D[42], fma(Lbar[40], D[41], fma(Lbar[39], D[40], fma(Lbar[38], D[39], fma(Lbar[37], D[38], fma(Lbar[36], D[37], fma(Lbar[35], D[36], fma(Lbar[34], D[35], fma(Lbar[33], D[34], fma(Lbar[32], D[33], fma(Lbar[31], D[32], fma(Lbar[30], D[31], fma(Lbar[29], D[30], fma(Lbar[28], D[29], fma(Lbar[27], D[28], fma(Lbar[26], D[27], fma(Lbar[25], D[26], fma(Lbar[24], D[25], fma(Lbar[23], D[24], fma(Lbar[22], D[23], fma(Lbar[21], D[22], fma(Lbar[20], D[21], fma(Lbar[19], D[20], fma(Lbar[18], D[19], fma(Lbar[17], D[18], fma(Lbar[16], D[17], fma(Lbar[15], D[16], fma(Lbar[14], D[15], fma(Lbar[13], D[14], fma(Lbar[12], D[13], fma(Lbar[11], D[12], fma(Lbar[10], D[11], fma(Lbar[9], D[10], fma(Lbar[8], D[9], fma(Lbar[7], D[8], fma(Lbar[6], D[7], fma(Lbar[5], D[6], fma(Lbar[4], D[5], fma(Lbar[3], D[4], fma(Lbar[2], D[3], fma(Lbar[1], D[2], Lbar[0] * D[1])))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))))), nu[0]);
  nu[1] = fma(T(-1), fma(Lbar[54], D[76], fma(Lbar[53], D[75], fma(Lbar[52], D[74], fma(Lbar[51], D[73], fma(Lbar[50], D[72], fma(Lbar[49], D[71], fma(Lbar[48], D[70], fma(Lbar[47], D[69], fma(Lbar[46], D[68], fma(Lbar[45], D[67], fma(Lbar[44], D[66], fma(Lbar[43], D[65], fma(Lbar[42], D[64], fma(Lbar[41], D[63], fma(Lbar[40], D[62], fma(Lbar[39], D[61], fma(Lbar[38], D[60], fma(Lbar[37], D[59], fma(Lbar[36], D[58], fma(Lbar[35], D[57], fma(Lbar[34], D[56], fma(Lbar[33], D[49], fma(Lbar[32], D[48], fma(Lbar[31], D[47], fma(Lbar[30], D[46], fma(Lbar[29], D[45], fma(Lbar[28], D[44], fma(Lbar[27], D[43], fma(Lbar[26], D[42], fma(Lbar[25], D[41], fma(Lbar[24], D[40], fma(Lbar[23], D[39], fma(Lbar[22], D[38], fma(Lbar[21], D[37], fma(Lbar[20], D[36], fma(Lbar[19], D[35], fma(Lbar[18], D[29], fma(Lbar[17], D[28], fma(Lbar[16], D[27], fma(Lbar[15], D[26], fma(Lbar[14], D[25], fma(Lbar[13], D[24], fma(Lbar[12], D[23], fma(Lbar[11], D[22], fma(Lbar[10], D[21], fma(Lbar[9], D[20], fma(Lbar[8], D[15], fma(Lbar[7], D[14], fma(Lbar[6], D[13], fma(Lbar[5], D[12], fma(Lbar[4], D[11], fma(Lbar[3], D[10], fma(Lbar[2], D[6], fma(Lbar[1], D[5], Lbar[0] * D[4])))))))))))))))))))))))))))))))))))))))))))))))))))))), nu[1]);
  nu[2] = fma(T(-1), fma(Lbar[54], D[82], fma(Lbar[53], D[81], fma(Lbar[52], D[80], fma(Lbar[51], D[79], fma(Lbar[50], D[78], fma(Lbar[49], D[77], fma(Lbar[48], D[75], fma(Lbar[47], D[74], fma(Lbar[46], D[73], fma(Lbar[45], D[72], fma(Lbar[44], D[71], fma(Lbar[43], D[69], fma(Lbar[42], D[68], fma(Lbar[41], D[67], fma(Lbar[40], D[66], fma(Lbar[39], D[64], fma(Lbar[38], D[63], fma(Lbar[37], D[62], fma(Lbar[36], D[60], fma(Lbar[35], D[59], fma(Lbar[34], D[57], fma(Lbar[33], D[54], fma(Lbar[32], D[53], fma(Lbar[31], D[52], fma(Lbar[30], D[51], fma(Lbar[29], D[50], fma(Lbar[28], D[48], fma(Lbar[27], D[47], fma(Lbar[26], D[46], fma(Lbar[25], D[45], fma(Lbar[24], D[43], fma(Lbar[23], D[42], fma(Lbar[22], D[41], fma(Lbar[21], D[39], fma(Lbar[20], D[38], fma(Lbar[19], D[36], fma(Lbar[18], D[33], fma(Lbar[17], D[32], fma(Lbar[16], D[31], fma(Lbar[15], D[30], fma(Lbar[14], D[28], fma(Lbar[13], D[27], fma(Lbar[12], D[26], fma(Lbar[11], D[24], fma(Lbar[10], D[23], fma(Lbar[9], D[21], fma(Lbar[8], D[18], fma(Lbar[7], D[17], fma(Lbar[6], D[16], fma(Lbar[5], D[14], fma(Lbar[4], D[13], fma(Lbar[3], D[11], fma(Lbar[2], D[8], fma(Lbar[1], D[7], Lbar[0] * D[5])))))))))))))))))))))))))))))))))))))))))))))))))))))), nu[2]);
  nu[3] = fma(T(-1), fma(Lbar[54], D[83], fma(Lbar[53], D[82], fma(Lbar[52], D[81], fma(Lbar[51], D[80], fma(Lbar[50], D[79], fma(Lbar[49], D[78], fma(Lbar[48], D[76], fma(Lbar[47], D[75], fma(Lbar[46], D[74], fma(Lbar[45], D[73], fma(Lbar[44], D[72], fma(Lbar[43], D[70], fma(Lbar[42], D[69], fma(Lbar[41], D[68], fma(Lbar[40], D[67], fma(Lbar[39], D[65], fma(Lbar[38], D[64], fma(Lbar[37], D[63], fma(Lbar[36], D[61], fma(Lbar[35], D[60], fma(Lbar[34], D[58], fma(Lbar[33], D[55], fma(Lbar[32], D[54], fma(Lbar[31], D[53], fma(Lbar[30], D[52], fma(Lbar[29], D[51], fma(Lbar[28], D[49], fma(Lbar[27], D[48], fma(Lbar[26], D[47], fma(Lbar[25], D[46], fma(Lbar[24], D[44], fma(Lbar[23], D[43], fma(Lbar[22], D[42], fma(Lbar[21], D[40], fma(Lbar[20], D[39], fma(Lbar[19], D[37], fma(Lbar[18], D[34], fma(Lbar[17], D[33], fma(Lbar[16], D[32], fma(Lbar[15], D[31], fma(Lbar[14], D[29], fma(Lbar[13], D[28], fma(Lbar[12], D[27], fma(Lbar[11], D[25], fma(Lbar[10], D[24], fma(Lbar[9], D[22], fma(Lbar[8], D[19], fma(Lbar[7], D[18], fma(Lbar[6], D[17], fma(Lbar[5], D[15], fma(Lbar[4], D[14], fma(Lbar[3], D[12], fma(Lbar[2], D[9], fma(Lbar[1], D[8], Lbar[0] * D[6])))))))))))))))))))))))))))))))))))))))))))))))))))))), nu[3]);
  nu[4] = fma(T(0.5), fma(Lbar[33], D[70], fma(Lbar[32], D[69], fma(Lbar[31], D[68], fma(Lbar[30], D[67], fma(Lbar[29], D[66], fma(Lbar[28], D[65], fma(Lbar[27], D[64], fma(Lbar[26], D[63], fma(Lbar[25], D[62], fma(Lbar[24], D[61], fma(Lbar[23], D[60], fma(Lbar[22], D[59], fma(Lbar[21], D[58], fma(Lbar[20], D[57], fma(Lbar[19], D[56], fma(Lbar[18], D[44], fma(Lbar[17], D[43], fma(Lbar[16], D[42], fma(Lbar[15], D[41], fma(Lbar[14], D[40], fma(Lbar[13], D[39], fma(Lbar[12], D[38], fma(Lbar[11], D[37], fma(Lbar[10], D[36], fma(Lbar[9], D[35], fma(Lbar[8], D[25], fma(Lbar[7], D[24], fma(Lbar[6], D[23], fma(Lbar[5], D[22], fma(Lbar[4], D[21], fma(Lbar[3], D[20], fma(Lbar[2], D[12], fma(Lbar[1], D[11], Lbar[0] * D[10]))))))))))))))))))))))))))))))))), nu[4]);
  nu[5] = fma(T(1), fma(Lbar[33], D[75], fma(Lbar[32], D[74], fma(Lbar[31], D[73], fma(Lbar[30], D[72], fma(Lbar[29], D[71], fma(Lbar[28], D[69], fma(Lbar[27], D[68], fma(Lbar[26], D[67], fma(Lbar[25], D[66], fma(Lbar[24], D[64], fma(Lbar[23], D[63], fma(Lbar[22], D[62], fma(Lbar[21], D[60], fma(Lbar[20], D[59], fma(Lbar[19], D[57], fma(Lbar[18], D[48], fma(Lbar[17], D[47], fma(Lbar[16], D[46], fma(Lbar[15], D[45], fma(Lbar[14], D[43], fma(Lbar[13], D[42], fma(Lbar[12], D[41], fma(Lbar[11], D[39], fma(Lbar[10], D[38], fma(Lbar[9], D[36], fma(Lbar[8], D[28], fma(Lbar[7], D[27], fma(Lbar[6], D[26], fma(Lbar[5], D[24], fma(Lbar[4], D[23], fma(Lbar[3], D[21], fma(Lbar[2], D[14], fma(Lbar[1], D[13], Lbar[0] * D[11]))))))))))))))))))))))))))))))))), nu[5]);
  nu[6] = fma(T(1), fma(Lbar[33], D[76], fma(Lbar[32], D[75], fma(Lbar[31], D[74], fma(Lbar[30], D[73], fma(Lbar[29], D[72], fma(Lbar[28], D[70], fma(Lbar[27], D[69], fma(Lbar[26], D[68], fma(Lbar[25], D[67], fma(Lbar[24], D[65], fma(Lbar[23], D[64], fma(Lbar[22], D[63], fma(Lbar[21], D[61], fma(Lbar[20], D[60], fma(Lbar[19], D[58], fma(Lbar[18], D[49], fma(Lbar[17], D[48], fma(Lbar[16], D[47], fma(Lbar[15], D[46], fma(Lbar[14], D[44], fma(Lbar[13], D[43], fma(Lbar[12], D[42], fma(Lbar[11], D[40], fma(Lbar[10], D[39], fma(Lbar[9], D[37], fma(Lbar[8], D[29], fma(Lbar[7], D[28], fma(Lbar[6], D[27], fma(Lbar[5], D[25], fma(Lbar[4], D[24], fma(Lbar[3], D[22], fma(Lbar[2], D[15], fma(Lbar[1], D[14], Lbar[0] * D[12]))))))))))))))))))))))))))))))))), nu[6]);
  nu[7] = fma(T(0.5), fma(Lbar[33], D[81], fma(Lbar[32], D[80], fma(Lbar[31], D[79], fma(Lbar[30], D[78], fma(Lbar[29], D[77], fma(Lbar[28], D[74], fma(Lbar[27], D[73], fma(Lbar[26], D[72], fma(Lbar[25], D[71], fma(Lbar[24], D[68], fma(Lbar[23], D[67], fma(Lbar[22], D[66], fma(Lbar[21], D[63], fma(Lbar[20], D[62], fma(Lbar[19], D[59], fma(Lbar[18], D[53], fma(Lbar[17], D[52], fma(Lbar[16], D[51], fma(Lbar[15], D[50], fma(Lbar[14], D[47], fma(Lbar[13], D[46], fma(Lbar[12], D[45], fma(Lbar[11], D[42], fma(Lbar[10], D[41], fma(Lbar[9], D[38], fma(Lbar[8], D[32], fma(Lbar[7], D[31], fma(Lbar[6], D[30], fma(Lbar[5], D[27], fma(Lbar[4], D[26], fma(Lbar[3], D[23], fma(Lbar[2], D[17], fma(Lbar[1], D[16], Lbar[0] * D[13]))))))))))))))))))))))))))))))))), nu[7]);
  nu[8] = fma(T(1), fma(Lbar[33], D[82], fma(Lbar[32], D[81], fma(Lbar[31], D[80], fma(Lbar[30], D[79], fma(Lbar[29], D[78], fma(Lbar[28], D[75], fma(Lbar[27], D[74], fma(Lbar[26], D[73], fma(Lbar[25], D[72], fma(Lbar[24], D[69], fma(Lbar[23], D[68], fma(Lbar[22], D[67], fma(Lbar[21], D[64], fma(Lbar[20], D[63], fma(Lbar[19], D[60], fma(Lbar[18], D[54], fma(Lbar[17], D[53], fma(Lbar[16], D[52], fma(Lbar[15], D[51], fma(Lbar[14], D[48], fma(Lbar[13], D[47], fma(Lbar[12], D[46], fma(Lbar[11], D[43], fma(Lbar[10], D[42], fma(Lbar[9], D[39], fma(Lbar[8], D[33], fma(Lbar[7], D[32], fma(Lbar[6], D[31], fma(Lbar[5], D[28], fma(Lbar[4], D[27], fma(Lbar[3], D[24], fma(Lbar[2], D[18], fma(Lbar[1], D[17], Lbar[0] * D[14]))))))))))))))))))))))))))))))))), nu[8]);
  nu[9] = fma(T(0.5), fma(Lbar[33], D[83], fma(Lbar[32], D[82], fma(Lbar[31], D[81], fma(Lbar[30], D[80], fma(Lbar[29], D[79], fma(Lbar[28], D[76], fma(Lbar[27], D[75], fma(Lbar[26], D[74], fma(Lbar[25], D[73], fma(Lbar[24], D[70], fma(Lbar[23], D[69], fma(Lbar[22], D[68], fma(Lbar[21], D[65], fma(Lbar[20], D[64], fma(Lbar[19], D[61], fma(Lbar[18], D[55], fma(Lbar[17], D[54], fma(Lbar[16], D[53], fma(Lbar[15], D[52], fma(Lbar[14], D[49], fma(Lbar[13], D[48], fma(Lbar[12], D[47], fma(Lbar[11], D[44], fma(Lbar[10], D[43], fma(Lbar[9], D[40], fma(Lbar[8], D[34], fma(Lbar[7], D[33], fma(Lbar[6], D[32], fma(Lbar[5], D[29], fma(Lbar[4], D[28], fma(Lbar[3], D[25], fma(Lbar[2], D[19], fma(Lbar[1], D[18], Lbar[0] * D[15]))))))))))))))))))))))))))))))))), nu[9]);
  nu[10] = fma(T(-0.16666666666666666), fma(Lbar[18], D[65], fma(Lbar[17], D[64], fma(Lbar[16], D[63], fma(Lbar[15], D[62], fma(Lbar[14], D[61], fma(Lbar[13], D[60], fma(Lbar[12], D[59], fma(Lbar[11], D[58], fma(Lbar[10], D[57], fma(Lbar[9], D[56], fma(Lbar[8], D[40], fma(Lbar[7], D[39], fma(Lbar[6], D[38], fma(Lbar[5], D[37], fma(Lbar[4], D[36], fma(Lbar[3], D[35], fma(Lbar[2], D[22], fma(Lbar[1], D[21], Lbar[0] * D[20])))))))))))))))))), nu[10]);
  nu[11] = fma(T(-0.5), fma(Lbar[18], D[69], fma(Lbar[17], D[68], fma(Lbar[16], D[67], fma(Lbar[15], D[66], fma(Lbar[14], D[64], fma(Lbar[13], D[63], fma(Lbar[12], D[62], fma(Lbar[11], D[60], fma(Lbar[10], D[59], fma(Lbar[9], D[57], fma(Lbar[8], D[43], fma(Lbar[7], D[42], fma(Lbar[6], D[41], fma(Lbar[5], D[39], fma(Lbar[4], D[38], fma(Lbar[3], D[36], fma(Lbar[2], D[24], fma(Lbar[1], D[23], Lbar[0] * D[21])))))))))))))))))), nu[11]);
  nu[12] = fma(T(-0.5), fma(Lbar[18], D[70], fma(Lbar[17], D[69], fma(Lbar[16], D[68], fma(Lbar[15], D[67], fma(Lbar[14], D[65], fma(Lbar[13], D[64], fma(Lbar[12], D[63], fma(Lbar[11], D[61], fma(Lbar[10], D[60], fma(Lbar[9], D[58], fma(Lbar[8], D[44], fma(Lbar[7], D[43], fma(Lbar[6], D[42], fma(Lbar[5], D[40], fma(Lbar[4], D[39], fma(Lbar[3], D[37], fma(Lbar[2], D[25], fma(Lbar[1], D[24], Lbar[0] * D[22])))))))))))))))))), nu[12]);
  nu[13] = fma(T(-0.5), fma(Lbar[18], D[74], fma(Lbar[17], D[73], fma(Lbar[16], D[72], fma(Lbar[15], D[71], fma(Lbar[14], D[68], fma(Lbar[13], D[67], fma(Lbar[12], D[66], fma(Lbar[11], D[63], fma(Lbar[10], D[62], fma(Lbar[9], D[59], fma(Lbar[8], D[47], fma(Lbar[7], D[46], fma(Lbar[6], D[45], fma(Lbar[5], D[42], fma(Lbar[4], D[41], fma(Lbar[3], D[38], fma(Lbar[2], D[27], fma(Lbar[1], D[26], Lbar[0] * D[23])))))))))))))))))), nu[13]);
  nu[14] = fma(T(-1), fma(Lbar[18], D[75], fma(Lbar[17], D[74], fma(Lbar[16], D[73], fma(Lbar[15], D[72], fma(Lbar[14], D[69], fma(Lbar[13], D[68], fma(Lbar[12], D[67], fma(Lbar[11], D[64], fma(Lbar[10], D[63], fma(Lbar[9], D[60], fma(Lbar[8], D[48], fma(Lbar[7], D[47], fma(Lbar[6], D[46], fma(Lbar[5], D[43], fma(Lbar[4], D[42], fma(Lbar[3], D[39], fma(Lbar[2], D[28], fma(Lbar[1], D[27], Lbar[0] * D[24])))))))))))))))))), nu[14]);
  nu[15] = fma(T(-0.5), fma(Lbar[18], D[76], fma(Lbar[17], D[75], fma(Lbar[16], D[74], fma(Lbar[15], D[73], fma(Lbar[14], D[70], fma(Lbar[13], D[69], fma(Lbar[12], D[68], fma(Lbar[11], D[65], fma(Lbar[10], D[64], fma(Lbar[9], D[61], fma(Lbar[8], D[49], fma(Lbar[7], D[48], fma(Lbar[6], D[47], fma(Lbar[5], D[44], fma(Lbar[4], D[43], fma(Lbar[3], D[40], fma(Lbar[2], D[29], fma(Lbar[1], D[28], Lbar[0] * D[25])))))))))))))))))), nu[15]);
  nu[16] = fma(T(-0.16666666666666666), fma(Lbar[18], D[80], fma(Lbar[17], D[79], fma(Lbar[16], D[78], fma(Lbar[15], D[77], fma(Lbar[14], D[73], fma(Lbar[13], D[72], fma(Lbar[12], D[71], fma(Lbar[11], D[67], fma(Lbar[10], D[66], fma(Lbar[9], D[62], fma(Lbar[8], D[52], fma(Lbar[7], D[51], fma(Lbar[6], D[50], fma(Lbar[5], D[46], fma(Lbar[4], D[45], fma(Lbar[3], D[41], fma(Lbar[2], D[31], fma(Lbar[1], D[30], Lbar[0] * D[26])))))))))))))))))), nu[16]);
  nu[17] = fma(T(-0.5), fma(Lbar[18], D[81], fma(Lbar[17], D[80], fma(Lbar[16], D[79], fma(Lbar[15], D[78], fma(Lbar[14], D[74], fma(Lbar[13], D[73], fma(Lbar[12], D[72], fma(Lbar[11], D[68], fma(Lbar[10], D[67], fma(Lbar[9], D[63], fma(Lbar[8], D[53], fma(Lbar[7], D[52], fma(Lbar[6], D[51], fma(Lbar[5], D[47], fma(Lbar[4], D[46], fma(Lbar[3], D[42], fma(Lbar[2], D[32], fma(Lbar[1], D[31], Lbar[0] * D[27])))))))))))))))))), nu[17]);
  nu[18] = fma(T(-0.5), fma(Lbar[18], D[82], fma(Lbar[17], D[81], fma(Lbar[16], D[80], fma(Lbar[15], D[79], fma(Lbar[14], D[75], fma(Lbar[13], D[74], fma(Lbar[12], D[73], fma(Lbar[11], D[69], fma(Lbar[10], D[68], fma(Lbar[9], D[64], fma(Lbar[8], D[54], fma(Lbar[7], D[53], fma(Lbar[6], D[52], fma(Lbar[5], D[48], fma(Lbar[4], D[47], fma(Lbar[3], D[43], fma(Lbar[2], D[33], fma(Lbar[1], D[32], Lbar[0] * D[28])))))))))))))))))), nu[18]);
  nu[19] = fma(T(-0.16666666666666666), fma(Lbar[18], D[83], fma(Lbar[17], D[82], fma(Lbar[16], D[81], fma(Lbar[15], D[80], fma(Lbar[14], D[76], fma(Lbar[13], D[75], fma(Lbar[12], D[74], fma(Lbar[11], D[70], fma(Lbar[10], D[69], fma(Lbar[9], D[65], fma(Lbar[8], D[55], fma(Lbar[7], D[54], fma(Lbar[6], D[53], fma(Lbar[5], D[49], fma(Lbar[4], D[48], fma(Lbar[3], D[44], fma(Lbar[2], D[34], fma(Lbar[1], D[33], Lbar[0] * D[29])))))))))))))))))), nu[19]);
  nu[20] = fma(T(0.041666666666666664), fma(Lbar[8], D[61], fma(Lbar[7], D[60], fma(Lbar[6], D[59], fma(Lbar[5], D[58], fma(Lbar[4], D[57], fma(Lbar[3], D[56], fma(Lbar[2], D[37], fma(Lbar[1], D[36], Lbar[0] * D[35])))))))), nu[20]);
  nu[21] = fma(T(0.16666666666666666), fma(Lbar[8], D[64], fma(Lbar[7], D[63], fma(Lbar[6], D[62], fma(Lbar[5], D[60], fma(Lbar[4], D[59], fma(Lbar[3], D[57], fma(Lbar[2], D[39], fma(Lbar[1], D[38], Lbar[0] * D[36])))))))), nu[21]);
  nu[22] = fma(T(0.16666666666666666), fma(Lbar[8], D[65], fma(Lbar[7], D[64], fma(Lbar[6], D[63], fma(Lbar[5], D[61], fma(Lbar[4], D[60], fma(Lbar[3], D[58], fma(Lbar[2], D[40], fma(Lbar[1], D[39], Lbar[0] * D[37])))))))), nu[22]);
  nu[23] = fma(T(0.25), fma(Lbar[8], D[68], fma(Lbar[7], D[67], fma(Lbar[6], D[66], fma(Lbar[5], D[63], fma(Lbar[4], D[62], fma(Lbar[3], D[59], fma(Lbar[2], D[42], fma(Lbar[1], D[41], Lbar[0] * D[38])))))))), nu[23]);
  nu[24] = fma(T(0.5), fma(Lbar[8], D[69], fma(Lbar[7], D[68], fma(Lbar[6], D[67], fma(Lbar[5], D[64], fma(Lbar[4], D[63], fma(Lbar[3], D[60], fma(Lbar[2], D[43], fma(Lbar[1], D[42], Lbar[0] * D[39])))))))), nu[24]);
  nu[25] = fma(T(0.25), fma(Lbar[8], D[70], fma(Lbar[7], D[69], fma(Lbar[6], D[68], fma(Lbar[5], D[65], fma(Lbar[4], D[64], fma(Lbar[3], D[61], fma(Lbar[2], D[44], fma(Lbar[1], D[43], Lbar[0] * D[40])))))))), nu[25]);
  nu[26] = fma(T(0.16666666666666666), fma(Lbar[8], D[73], fma(Lbar[7], D[72], fma(Lbar[6], D[71], fma(Lbar[5], D[67], fma(Lbar[4], D[66], fma(Lbar[3], D[62], fma(Lbar[2], D[46], fma(Lbar[1], D[45], Lbar[0] * D[41])))))))), nu[26]);
  nu[27] = fma(T(0.5), fma(Lbar[8], D[74], fma(Lbar[7], D[73], fma(Lbar[6], D[72], fma(Lbar[5], D[68], fma(Lbar[4], D[67], fma(Lbar[3], D[63], fma(Lbar[2], D[47], fma(Lbar[1], D[46], Lbar[0] * D[42])))))))), nu[27]);
  nu[28] = fma(T(0.5), fma(Lbar[8], D[75], fma(Lbar[7], D[74], fma(Lbar[6], D[73], fma(Lbar[5], D[69], fma(Lbar[4], D[68], fma(Lbar[3], D[64], fma(Lbar[2], D[48], fma(Lbar[1], D[47], Lbar[0] * D[43])))))))), nu[28]);
  nu[29] = fma(T(0.16666666666666666), fma(Lbar[8], D[76], fma(Lbar[7], D[75], fma(Lbar[6], D[74], fma(Lbar[5], D[70], fma(Lbar[4], D[69], fma(Lbar[3], D[65], fma(Lbar[2], D[49], fma(Lbar[1], D[48], Lbar[0] * D[44])))))))), nu[29]);
  nu[30] = fma(T(0.041666666666666664), fma(Lbar[8], D[79], fma(Lbar[7], D[78], fma(Lbar[6], D[77], fma(Lbar[5], D[72], fma(Lbar[4], D[71], fma(Lbar[3], D[66], fma(Lbar[2], D[51], fma(Lbar[1], D[50], Lbar[0] * D[45])))))))), nu[30]);
  nu[31] = fma(T(0.16666666666666666), fma(Lbar[8], D[80], fma(Lbar[7], D[79], fma(Lbar[6], D[78], fma(Lbar[5], D[73], fma(Lbar[4], D[72], fma(Lbar[3], D[67], fma(Lbar[2], D[52], fma(Lbar[1], D[51], Lbar[0] * D[46])))))))), nu[31]);
  nu[32] = fma(T(0.25), fma(Lbar[8], D[81], fma(Lbar[7], D[80], fma(Lbar[6], D[79], fma(Lbar[5], D[74], fma(Lbar[4], D[73], fma(Lbar[3], D[68], fma(Lbar[2], D[53], fma(Lbar[1], D[52], Lbar[0] * D[47])))))))), nu[32]);
  nu[33] = fma(T(0.16666666666666666), fma(Lbar[8], D[82], fma(Lbar[7], D[81], fma(Lbar[6], D[80], fma(Lbar[5], D[75], fma(Lbar[4], D[74], fma(Lbar[3], D[69], fma(Lbar[2], D[54], fma(Lbar[1], D[53], Lbar[0] * D[48])))))))), nu[33]);
  nu[34] = fma(T(0.041666666666666664), fma(Lbar[8], D[83], fma(Lbar[7], D[82], fma(Lbar[6], D[81], fma(Lbar[5], D[76], fma(Lbar[4], D[75], fma(Lbar[3], D[70], fma(Lbar[2], D[55], fma(Lbar[1], D[54], Lbar[0] * D[49])))))))), nu[34]);
  nu[35] = fma(T(-0.0083333333333333332), fma(Lbar[2], D[58], fma(Lbar[1], D[57], Lbar[0] * D[56])), nu[35]);
  nu[36] = fma(T(-0.041666666666666664), fma(Lbar[2], D[60], fma(Lbar[1], D[59], Lbar[0] * D[57])), nu[36]);
  nu[37] = fma(T(-0.041666666666666664), fma(Lbar[2], D[61], fma(Lbar[1], D[60], Lbar[0] * D[58])), nu[37]);
  nu[38] = fma(T(-0.083333333333333329), fma(Lbar[2], D[63], fma(Lbar[1], D[62], Lbar[0] * D[59])), nu[38]);
  nu[39] = fma(T(-0.16666666666666666), fma(Lbar[2], D[64], fma(Lbar[1], D[63], Lbar[0] * D[60])), nu[39]);
  nu[40] = fma(T(-0.083333333333333329), fma(Lbar[2], D[65], fma(Lbar[1], D[64], Lbar[0] * D[61])), nu[40]);
  nu[41] = fma(T(-0.083333333333333329), fma(Lbar[2], D[67], fma(Lbar[1], D[66], Lbar[0] * D[62])), nu[41]);
  nu[42] = fma(T(-0.25), fma(Lbar[2], D[68], fma(Lbar[1], D[67], Lbar[0] * D[63])), nu[42]);
  nu[43] = fma(T(-0.25), fma(Lbar[2], D[69], fma(Lbar[1], D[68], Lbar[0] * D[64])), nu[43]);
  nu[44] = fma(T(-0.083333333333333329), fma(Lbar[2], D[70], fma(Lbar[1], D[69], Lbar[0] * D[65])), nu[44]);
  nu[45] = fma(T(-0.041666666666666664), fma(Lbar[2], D[72], fma(Lbar[1], D[71], Lbar[0] * D[66])), nu[45]);
  nu[46] = fma(T(-0.16666666666666666), fma(Lbar[2], D[73], fma(Lbar[1], D[72], Lbar[0] * D[67])), nu[46]);
  nu[47] = fma(T(-0.25), fma(Lbar[2], D[74], fma(Lbar[1], D[73], Lbar[0] * D[68])), nu[47]);
  nu[48] = fma(T(-0.16666666666666666), fma(Lbar[2], D[75], fma(Lbar[1], D[74], Lbar[0] * D[69])), nu[48]);
  nu[49] = fma(T(-0.041666666666666664), fma(Lbar[2], D[76], fma(Lbar[1], D[75], Lbar[0] * D[70])), nu[49]);
  nu[50] = fma(T(-0.0083333333333333332), fma(Lbar[2], D[78], fma(Lbar[1], D[77], Lbar[0] * D[71])), nu[50]);
  nu[51] = fma(T(-0.041666666666666664), fma(Lbar[2], D[79], fma(Lbar[1], D[78], Lbar[0] * D[72])), nu[51]);
  nu[52] = fma(T(-0.083333333333333329), fma(Lbar[2], D[80], fma(Lbar[1], D[79], Lbar[0] * D[73])), nu[52]);
  nu[53] = fma(T(-0.083333333333333329), fma(Lbar[2], D[81], fma(Lbar[1], D[80], Lbar[0] * D[74])), nu[53]);
  nu[54] = fma(T(-0.041666666666666664), fma(Lbar[2], D[82], fma(Lbar[1], D[81], Lbar[0] * D[75])), nu[54]);
  nu[55] = fma(T(-0.0083333333333333332), fma(Lbar[2], D[83], fma(Lbar[1], D[82], Lbar[0] * D[76])), nu[55]);
}

