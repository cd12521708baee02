// Cloud-in-cell density contrast and the loss L = sum_c delta_c^2 with its
// gradient with respect to the particle positions (the loss of the
// differentiable trajectory; not in the paper).  Cell c of an ng^3 grid has
// its centre at (c + 1/2)/ng; rho_c = ng^3 sum_j m_j w_jc, delta = rho - 1.
#include "common.cuh"

namespace {

__device__ __forceinline__ void cic_axis(double x, int ng, int& i0, double& f) {
  const double u = x * ng - 0.5;
  const double fl = floor(u);
  f = u - fl;
  long long i = (long long)fl;
  i %= ng;
  if (i < 0) i += ng;
  i0 = (int)i;
}

__global__ void cic_deposit_kernel(int64_t n, const double* __restrict__ pos, const float* __restrict__ mass, int ng,
                                   double* __restrict__ grid) {
  const double scale = (double)ng * ng * ng;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; d++) cic_axis(pos[d * n + j], ng, i0[d], f[d]);
    const double m = (mass ? (double)mass[j] : 1.0 / (double)n) * scale;
    for (int c = 0; c < 8; c++) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
      const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
      const int ix = (i0[0] + dx) % ng, iy = (i0[1] + dy) % ng, iz = (i0[2] + dz) % ng;
      atomicAdd(&grid[((int64_t)ix * ng + iy) * ng + iz], m * w);
    }
  }
}

__global__ void cic_loss_kernel(int64_t ncell, double* __restrict__ grid, double* __restrict__ loss) {
  double s = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    const double d = grid[c] - 1.0;
    grid[c] = d;  // the grid now holds delta
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

__global__ void cic_grad_kernel(int64_t n, const double* __restrict__ pos, const float* __restrict__ mass, int ng,
                                const double* __restrict__ delta, double* __restrict__ grad) {
  const double scale = (double)ng * ng * ng;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; d++) cic_axis(pos[d * n + j], ng, i0[d], f[d]);
    const double m = (mass ? (double)mass[j] : 1.0 / (double)n) * scale;
    double g[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 8; c++) {
      const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
      const double wx = dx ? f[0] : 1.0 - f[0], wy = dy ? f[1] : 1.0 - f[1], wz = dz ? f[2] : 1.0 - f[2];
      const int ix = (i0[0] + dx) % ng, iy = (i0[1] + dy) % ng, iz = (i0[2] + dz) % ng;
      const double v = 2.0 * delta[((int64_t)ix * ng + iy) * ng + iz] * m;
      const double sx = dx ? ng : -ng, sy = dy ? ng : -ng, sz = dz ? ng : -ng;
      g[0] += v * sx * wy * wz;
      g[1] += v * wx * sy * wz;
      g[2] += v * wx * wy * sz;
    }
    for (int d = 0; d < 3; d++) grad[d * n + j] = g[d];
  }
}

// Zel'dovich state of the trajectory's start: x = q + a psi wrapped into
// [0, 1), p = H0 a^(3/2) psi (growing mode of the comoving equations, D = a)
__global__ void zeldovich_state_kernel(int64_t n3, const double* __restrict__ q, const double* __restrict__ psi,
                                       double a, double pa, double* __restrict__ pos, float* __restrict__ mom) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
    const double u = psi[i];
    double x = __dadd_rn(q[i], __dmul_rn(a, u));  // rounded as written, no contraction
    x -= floor(x);
    pos[i] = x < 1.0 ? x : 0.0;
    mom[i] = (float)(pa * u);
  }
}

// its transpose: d psi = a lam_x + H0 a^(3/2) lam_p (the wrap has unit slope)
__global__ void zeldovich_vjp_kernel(int64_t n3, double a, double pa, const double* __restrict__ lx,
                                     const float* __restrict__ lp, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __dadd_rn(__dmul_rn(a, lx[i]), __dmul_rn(pa, (double)lp[i]));
}

int gridc(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

extern "C" int nbody_cic_loss(const double* pos_dev, const float* mass_dev, int64_t n, int ng, double* grid_dev,
                              double* loss_dev, double* grad_dev, nbody_stream_t stream) {
  if (!pos_dev || !grid_dev || !loss_dev || n <= 0 || ng < 2 || ng > 1024) return NBODY_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ncell = (int64_t)ng * ng * ng;
  if (cudaMemsetAsync(grid_dev, 0, sizeof(double) * ncell, s) != cudaSuccess) return NBODY_ECUDA;
  if (cudaMemsetAsync(loss_dev, 0, sizeof(double), s) != cudaSuccess) return NBODY_ECUDA;
  cic_deposit_kernel<<<gridc(n, 256), 256, 0, s>>>(n, pos_dev, mass_dev, ng, grid_dev);
  cic_loss_kernel<<<gridc(ncell, 256), 256, 0, s>>>(ncell, grid_dev, loss_dev);
  nb_launch_counter += 2;
  if (grad_dev) {
    cic_grad_kernel<<<gridc(n, 256), 256, 0, s>>>(n, pos_dev, mass_dev, ng, grid_dev, grad_dev);
    nb_launch_counter += 1;
  }
  return cudaGetLastError() == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

extern "C" int nbody_zeldovich_state(int64_t n, const double* q_dev, const double* psi_dev, double a,
                                     double* pos_dev, float* mom_dev, nbody_stream_t stream) {
  if (!q_dev || !psi_dev || !pos_dev || !mom_dev || n <= 0 || !(a > 0.0) || !(a < 1e300)) return NBODY_EINVAL;
  const double pa = sqrt(8.0 * M_PI / 3.0) * a * sqrt(a);
  zeldovich_state_kernel<<<gridc(3 * n, 256), 256, 0, (cudaStream_t)stream>>>(3 * n, q_dev, psi_dev, a, pa,
                                                                               pos_dev, mom_dev);
  nb_launch_counter += 1;
  return cudaGetLastError() == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}

extern "C" int nbody_zeldovich_vjp(int64_t n, double a, const double* lam_pos_dev, const float* lam_mom_dev,
                                   double* dpsi_dev, nbody_stream_t stream) {
  if (!lam_pos_dev || !lam_mom_dev || !dpsi_dev || n <= 0 || !(a > 0.0) || !(a < 1e300)) return NBODY_EINVAL;
  const double pa = sqrt(8.0 * M_PI / 3.0) * a * sqrt(a);
  zeldovich_vjp_kernel<<<gridc(3 * n, 256), 256, 0, (cudaStream_t)stream>>>(3 * n, a, pa, lam_pos_dev, lam_mom_dev,
                                                                             dpsi_dev);
  nb_launch_counter += 1;
  return cudaGetLastError() == cudaSuccess ? NBODY_OK : NBODY_ECUDA;
}
