// Particle kernels of the SIPF-PIC step: the move of Algorithm 4 (noise,
// gather of grad c with I* (Algorithm 3), drift, periodic wrap) fused with the
// deposit I of the new positions (Algorithm 2), plus the stand-alone deposit,
// gather, noise and FP64 reduction kernels.
#include <cuda_runtime.h>
#include <math.h>

#include "sipf_internal.h"

namespace sipf {

template <typename T> Geo<T> make_geo(double L, int H) {
  Geo<T> g;
  g.L = (T)L;
  g.invL = (T)(1.0 / L);
  g.half_L = (T)(0.5 * L);
  g.inv_h = (T)((double)H / L);
  g.H = H;
  g.mask = H - 1;
  return g;
}
template Geo<float> make_geo<float>(double, int);
template Geo<double> make_geo<double>(double, int);

static inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > (1LL << 30)) b = 1LL << 30;
  if (b < 1) b = 1;
  return (int)b;
}

// Deposit one particle's stencil into the grid: floating-point reductions, or
// 64-bit fixed point (w already holds 2^60 / P) for a result that does not
// depend on the order of the additions.
template <typename T>
__device__ __forceinline__ void deposit_one(void* phi, int fixed, int order, T px, T py, T pz, const Geo<T>& g,
                                            T w) {
  int cx, cy, cz;
  T lx, ly, lz;
  cell_lambda(px, g, cx, lx);
  cell_lambda(py, g, cy, ly);
  cell_lambda(pz, g, cz, lz);
  if (!fixed) {
    T* grid = static_cast<T*>(phi);
    stencil_visit<T>(order, cx, cy, cz, lx, ly, lz, g.H, g.mask,
                     [&](int idx, T f) { atomicAdd(grid + idx, w * f); });
  } else {
    unsigned long long* acc = static_cast<unsigned long long*>(phi);
    stencil_visit<T>(order, cx, cy, cz, lx, ly, lz, g.H, g.mask, [&](int idx, T f) {
      const long long v = (long long)llrint((double)(w * f));
      atomicAdd(acc + idx, (unsigned long long)v);
    });
  }
}

template <typename T> struct V3 { T x, y, z; };
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ V3<float> load(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z};
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ V3<double> load(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double b = __ldg(p + 2);
    return {a.x, a.y, b};
  }
};

// Gather of the three gradient components (interleaved 4-wide nodes) at (px,py,pz).
template <typename T>
__device__ __forceinline__ void gather_grad(const T* grad4, int order, T px, T py, T pz, const Geo<T>& g, T& gx,
                                            T& gy, T& gz) {
  int cx, cy, cz;
  T lx, ly, lz;
  cell_lambda(px, g, cx, lx);
  cell_lambda(py, g, cy, ly);
  cell_lambda(pz, g, cz, lz);
  T ax = 0, ay = 0, az = 0;
  stencil_visit<T>(order, cx, cy, cz, lx, ly, lz, g.H, g.mask, [&](int idx, T f) {
    const auto v = Vec4<T>::load(grad4 + (size_t)idx * 4);
    ax += f * v.x;
    ay += f * v.y;
    az += f * v.z;
  });
  gx = ax;
  gy = ay;
  gz = az;
}

// One thread per particle: X^{n-1} -> X^n (Algorithm 4, particle loop), then
// deposit X^n for the next step's F_H I(rho-hat^(n)).
template <typename T>
__global__ void __launch_bounds__(256) k_move_deposit(MoveArgs<T> a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.P; p += stride) {
    const T x = a.x[p], y = a.y[p], z = a.z[p];
    T nz[6];
    normals6(a.seed, (uint64_t)p, a.n, nz);
    T nx, ny, nw;
    if (a.split == 0) {
      // Z = X + W^- + chi tau I*(grad c)(X + W^-),  X^n = Z + W^+
      const T yx = x + a.s_noise * nz[0], yy = y + a.s_noise * nz[1], yz = z + a.s_noise * nz[2];
      T gx, gy, gz;
      gather_grad(a.grad4, a.g2p, yx, yy, yz, a.g, gx, gy, gz);
      nx = wrap_coord((yx + a.chitau * gx) + a.s_noise * nz[3], a.g);
      ny = wrap_coord((yy + a.chitau * gy) + a.s_noise * nz[4], a.g);
      nw = wrap_coord((yz + a.chitau * gz) + a.s_noise * nz[5], a.g);
    } else {
      // X^n = X + chi tau I*(grad c)(X) + W,  W ~ N(0, 2 mu tau I)
      T gx, gy, gz;
      gather_grad(a.grad4, a.g2p, x, y, z, a.g, gx, gy, gz);
      nx = wrap_coord((x + a.chitau * gx) + a.s_noise * nz[0], a.g);
      ny = wrap_coord((y + a.chitau * gy) + a.s_noise * nz[1], a.g);
      nw = wrap_coord((z + a.chitau * gz) + a.s_noise * nz[2], a.g);
    }
    a.x[p] = nx;
    a.y[p] = ny;
    a.z[p] = nw;
    if (!(t_finite(nx) && t_finite(ny) && t_finite(nw))) atomicOr(a.err, 1);
    deposit_one<T>(a.phi, a.fixed, a.p2g, nx, ny, nw, a.g, a.w);
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_deposit(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, Geo<T> g, T w,
          void* phi, int order, int fixed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride)
    deposit_one<T>(phi, fixed, order, x[p], y[p], z[p], g, w);
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gather(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, Geo<T> g,
         const T* __restrict__ f, int ncomp, int interleaved4, int order, T* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const size_t N = (size_t)g.H * g.H * g.H;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    int cx, cy, cz;
    T lx, ly, lz;
    cell_lambda(x[p], g, cx, lx);
    cell_lambda(y[p], g, cy, ly);
    cell_lambda(z[p], g, cz, lz);
    for (int c = 0; c < ncomp; ++c) {
      T acc = 0;
      stencil_visit<T>(order, cx, cy, cz, lx, ly, lz, g.H, g.mask, [&](int idx, T wt) {
        acc += wt * (interleaved4 ? f[(size_t)idx * 4 + c] : f[c * N + idx]);
      });
      out[(size_t)c * P + p] = acc;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_noise(uint64_t seed, uint32_t step, int64_t first, int64_t P, T* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    T v[6];
    normals6(seed, (uint64_t)(first + p), step, v);
#pragma unroll
    for (int j = 0; j < 6; ++j) z[(size_t)j * P + p] = v[j];
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc2[0] += sum |X|^2, acc2[1] += sum sqrt(x^2 + y^2)  (FP64)
template <typename T>
__global__ void __launch_bounds__(256)
k_moments(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, double* acc2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double s2 = 0.0, sr = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    const double a = x[p], b = y[p], c = z[p];
    s2 += a * a + b * b + c * c;
    sr += sqrt(a * a + b * b);
  }
  s2 = warp_sum(s2);
  sr = warp_sum(sr);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc2, s2);
    atomicAdd(acc2 + 1, sr);
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_aos_to_soa(const double* __restrict__ aos, int64_t P, Geo<T> g, T* x, T* y, T* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    x[p] = wrap_coord((T)aos[3 * p + 0], g);
    y[p] = wrap_coord((T)aos[3 * p + 1], g);
    z[p] = wrap_coord((T)aos[3 * p + 2], g);
  }
}

// acc2[0] += sum_q mult |alpha_q|^2 over ||q|| >= 4, acc2[1] += the full sum
// (mult = 2 for 0 < kz < H/2 accounts for the Hermitian partner).
template <typename T>
__global__ void __launch_bounds__(256) k_alpha_energy(const cpx<T>* __restrict__ alpha, int H, double* acc2) {
  const int nh = H / 2 + 1;
  const int64_t n = (int64_t)H * H * nh;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double hi = 0.0, tot = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int kz = (int)(i % nh);
    const int ky = (int)((i / nh) % H);
    const int kx = (int)(i / ((int64_t)nh * H));
    const int qx = kx < H / 2 ? kx : kx - H, qy = ky < H / 2 ? ky : ky - H, qz = kz < H / 2 ? kz : kz - H;
    const double mult = (kz == 0 || kz == H / 2) ? 1.0 : 2.0;
    const cpx<T> a = alpha[i];
    const double e = mult * ((double)a.x * a.x + (double)a.y * a.y);
    tot += e;
    if (qx * qx + qy * qy + qz * qz >= 16) hi += e;
  }
  hi = warp_sum(hi);
  tot = warp_sum(tot);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc2, hi);
    atomicAdd(acc2 + 1, tot);
  }
}

// ---------------------------------------------------------------------------
template <typename T> cudaError_t launch_move_deposit(const MoveArgs<T>& a, cudaStream_t s) {
  k_move_deposit<T><<<grid_for(a.P, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, T w, void* phi, int order,
                           int fixed, cudaStream_t s) {
  k_deposit<T><<<grid_for(P, 256), 256, 0, s>>>(x, y, z, P, g, w, phi, order, fixed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, const T* f, int ncomp,
                          int interleaved4, int order, T* out, cudaStream_t s) {
  k_gather<T><<<grid_for(P, 256), 256, 0, s>>>(x, y, z, P, g, f, ncomp, interleaved4, order, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_noise(uint64_t seed, int64_t step, int64_t first, int64_t P, T* z, cudaStream_t s) {
  k_noise<T><<<grid_for(P, 256), 256, 0, s>>>(seed, (uint32_t)step, first, P, z);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const T* x, const T* y, const T* z, int64_t P, double* acc2, cudaStream_t s) {
  int b = grid_for(P, 256);
  if (b > 152 * 8) b = 152 * 8;
  k_moments<T><<<b, 256, 0, s>>>(x, y, z, P, acc2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_aos_to_soa(const double* aos, int64_t P, Geo<T> g, T* x, T* y, T* z, cudaStream_t s) {
  k_aos_to_soa<T><<<grid_for(P, 256), 256, 0, s>>>(aos, P, g, x, y, z);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_alpha_energy(const cpx<T>* alpha, int H, double* acc2, cudaStream_t s) {
  const int64_t n = (int64_t)H * H * (H / 2 + 1);
  int b = grid_for(n, 256);
  if (b > 152 * 8) b = 152 * 8;
  k_alpha_energy<T><<<b, 256, 0, s>>>(alpha, H, acc2);
  return cudaGetLastError();
}

#define SIPF_INST(T)                                                                                          \
  template cudaError_t launch_move_deposit<T>(const MoveArgs<T>&, cudaStream_t);                              \
  template cudaError_t launch_deposit<T>(const T*, const T*, const T*, int64_t, Geo<T>, T, void*, int, int,   \
                                         cudaStream_t);                                                      \
  template cudaError_t launch_gather<T>(const T*, const T*, const T*, int64_t, Geo<T>, const T*, int, int,   \
                                        int, T*, cudaStream_t);                                              \
  template cudaError_t launch_noise<T>(uint64_t, int64_t, int64_t, int64_t, T*, cudaStream_t);               \
  template cudaError_t launch_moments<T>(const T*, const T*, const T*, int64_t, double*, cudaStream_t);      \
  template cudaError_t launch_aos_to_soa<T>(const double*, int64_t, Geo<T>, T*, T*, T*, cudaStream_t);       \
  template cudaError_t launch_alpha_energy<T>(const cpx<T>*, int, double*, cudaStream_t);
SIPF_INST(float)
SIPF_INST(double)
#undef SIPF_INST

}  // namespace sipf
