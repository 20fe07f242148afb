// Reverse-mode (adjoint) kernels of the SIPF-PIC step with the noise held
// fixed: the transposes of the deposit I (Algorithm 2), of the gather I*
// (Algorithm 3) and of the Fourier-side update (Eq. (alpha_hat_update), the
// filtered spectral gradient of Algorithm 4), and the position derivatives of
// the weight polynomials of Eqs. (2ord) and (4ord).  The reverse step takes
// the particles in the order of the forward step's tile bins (consecutive
// entries share a grid tile, so the gathers and the cotangent reductions stay
// local), each entry carrying its particle id; Xbar is kept per particle as a
// 4-wide record (one vector load and store per entry).  The gradient and
// cotangent grids are small enough to stay in L2 at the sizes the adjoint
// serves.
#include <cuda_runtime.h>

#include "sipf_device.cuh"
#include "sipf_internal.h"

namespace sipf {
namespace {

template <typename T> struct A3 { T x, y, z; };

// 1D factors and their derivatives on one axis: in-cell layers j = 0, 1 and
// the outer layers -1 (om) and 2 (o2) of Gamma_4.
template <typename T> struct AxisD {
  T f[2], d[2];     // 1 - l, l and -1, +1
  T om, dom, o2, do2;
  T q, dq;          // l (1 - l) / 2 and its derivative (the boost term of the inner nodes)
};

template <typename T> __device__ __forceinline__ AxisD<T> axis_d(T l) {
  AxisD<T> a;
  a.f[0] = T(1) - l;
  a.f[1] = l;
  a.d[0] = T(-1);
  a.d[1] = T(1);
  const T s6 = T(1.0 / 6.0);
  a.om = -(T(2) - l) * l * (T(1) - l) * s6;           // -(2 l - 3 l^2 + l^3) / 6
  a.dom = -(T(2) - T(6) * l + T(3) * l * l) * s6;
  a.o2 = -(T(1) + l) * (T(1) - l) * l * s6;           // -(l - l^3) / 6
  a.do2 = -(T(1) - T(3) * l * l) * s6;
  a.q = T(0.5) * l * (T(1) - l);
  a.dq = T(0.5) * (T(1) - T(2) * l);
  return a;
}

// Visit the 8 nodes of Gamma_2 with F and dF/dlambda: fn(idx, F, Fx, Fy, Fz).
template <typename T, typename Fn>
__device__ __forceinline__ void gamma2_grad_visit(const int ix[4], const int iy[4], const int iz[4], const AxisD<T>& ax,
                                                  const AxisD<T>& ay, const AxisD<T>& az, Fn&& fn) {
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        fn(ix[a + 1] + iy[b + 1] + iz[c + 1], ax.f[a] * ay.f[b] * az.f[c], ax.d[a] * ay.f[b] * az.f[c],
           ax.f[a] * ay.d[b] * az.f[c], ax.f[a] * ay.f[b] * az.d[c]);
}

// Visit the 32 nodes of Gamma_4 with F and dF/dlambda.  Inner nodes:
// F = B(l) prod f, B = 1 + sum_k l_k (1 - l_k)/2; outer nodes: the cubic factor
// of their axis times the bilinear factor of the other two.
template <typename T, typename Fn>
__device__ __forceinline__ void gamma4_grad_visit(const int ix[4], const int iy[4], const int iz[4], const AxisD<T>& ax,
                                                  const AxisD<T>& ay, const AxisD<T>& az, Fn&& fn) {
  const T B = T(1) + ax.q + ay.q + az.q;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T tri = ax.f[a] * ay.f[b] * az.f[c];
        fn(ix[a + 1] + iy[b + 1] + iz[c + 1], B * tri, ax.dq * tri + B * ax.d[a] * ay.f[b] * az.f[c],
           ay.dq * tri + B * ax.f[a] * ay.d[b] * az.f[c], az.dq * tri + B * ax.f[a] * ay.f[b] * az.d[c]);
      }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T yz = ay.f[b] * az.f[c];
      fn(ix[0] + iy[b + 1] + iz[c + 1], ax.om * yz, ax.dom * yz, ax.om * ay.d[b] * az.f[c], ax.om * ay.f[b] * az.d[c]);
      fn(ix[3] + iy[b + 1] + iz[c + 1], ax.o2 * yz, ax.do2 * yz, ax.o2 * ay.d[b] * az.f[c], ax.o2 * ay.f[b] * az.d[c]);
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T xz = ax.f[a] * az.f[c];
      fn(ix[a + 1] + iy[0] + iz[c + 1], ay.om * xz, ay.om * ax.d[a] * az.f[c], ay.dom * xz, ay.om * ax.f[a] * az.d[c]);
      fn(ix[a + 1] + iy[3] + iz[c + 1], ay.o2 * xz, ay.o2 * ax.d[a] * az.f[c], ay.do2 * xz, ay.o2 * ax.f[a] * az.d[c]);
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T xy = ax.f[a] * ay.f[b];
      fn(ix[a + 1] + iy[b + 1] + iz[0], az.om * xy, az.om * ax.d[a] * ay.f[b], az.om * ax.f[a] * ay.d[b], az.dom * xy);
      fn(ix[a + 1] + iy[b + 1] + iz[3], az.o2 * xy, az.o2 * ax.d[a] * ay.f[b], az.o2 * ax.f[a] * ay.d[b], az.do2 * xy);
    }
}

template <typename T, typename Fn>
__device__ __forceinline__ void stencil_grad_visit(int order, T px, T py, T pz, const Geo<T>& g, Fn&& fn) {
  int cx, cy, cz;
  T lx, ly, lz;
  cell_lambda(px, g, cx, lx);
  cell_lambda(py, g, cy, ly);
  cell_lambda(pz, g, cz, lz);
  int ix[4], iy[4], iz[4];
  axis_layers_global(cx, g.mask, g.H * g.H, ix);
  axis_layers_global(cy, g.mask, g.H, iy);
  axis_layers_global(cz, g.mask, 1, iz);
  const AxisD<T> ax = axis_d(lx), ay = axis_d(ly), az = axis_d(lz);
  if (order == 4) gamma4_grad_visit<T>(ix, iy, iz, ax, ay, az, fn);
  else gamma2_grad_visit<T>(ix, iy, iz, ax, ay, az, fn);
}

// w (H/L) sum_gamma grad_lambda F_gamma(lambda(X)) phibar[q_gamma]: the
// transpose of X -> I rho-hat(X) applied to the grid cotangent phibar.
template <typename T>
__device__ __forceinline__ A3<T> deposit_adjoint(const T* __restrict__ phibar, int order, T px, T py, T pz, T w_inv_h,
                                                 const Geo<T>& g) {
  A3<T> s{T(0), T(0), T(0)};
  stencil_grad_visit<T>(order, px, py, pz, g, [&](int idx, T, T fx, T fy, T fz) {
    const T f = __ldg(phibar + idx);
    s.x += fx * f;
    s.y += fy * f;
    s.z += fz * f;
  });
  return A3<T>{s.x * w_inv_h, s.y * w_inv_h, s.z * w_inv_h};
}

// The same for Gamma_4 from the z-quads of phibar (quad at node (x, y, z):
// phibar at z - 1, z, z + 1, z + 2): the 32 nodes lie on 12 (x, y) columns,
// the four inner columns using all four z layers (the z-outer nodes and the
// inner ones), the x-outer and y-outer columns the two inner z layers; one
// vector load per column instead of one scalar load per node.
template <typename T> struct Quad { T v[4]; };
template <typename T> __device__ __forceinline__ Quad<T> load_quad(const T* p);
template <> __device__ __forceinline__ Quad<float> load_quad<float>(const float* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {{v.x, v.y, v.z, v.w}};
}
template <> __device__ __forceinline__ Quad<double> load_quad<double>(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {{a.x, a.y, b.x, b.y}};
}

template <typename T>
__device__ __forceinline__ A3<T> deposit_adjoint4_quads(const T* __restrict__ quads, T px, T py, T pz, T w_inv_h,
                                                        const Geo<T>& g) {
  int cx, cy, cz;
  T lx, ly, lz;
  cell_lambda(px, g, cx, lx);
  cell_lambda(py, g, cy, ly);
  cell_lambda(pz, g, cz, lz);
  int ix[4], iy[4];
  axis_layers_global(cx, g.mask, g.H * g.H, ix);
  axis_layers_global(cy, g.mask, g.H, iy);
  const int iz = cz & g.mask;
  const AxisD<T> ax = axis_d(lx), ay = axis_d(ly), az = axis_d(lz);
  const T B = T(1) + ax.q + ay.q + az.q;
  A3<T> s{T(0), T(0), T(0)};
  auto add = [&](T fx, T fy, T fz, T v) {
    s.x += fx * v;
    s.y += fy * v;
    s.z += fz * v;
  };
  // inner columns: z-outer node (layer 0, om), inner nodes (layers 1, 2), z-outer node (layer 3, o2)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const Quad<T> q = load_quad<T>(quads + (size_t)(ix[a + 1] + iy[b + 1] + iz) * 4);
      const T fxy = ax.f[a] * ay.f[b], dxy = ax.d[a] * ay.f[b], xdy = ax.f[a] * ay.d[b];
      add(az.om * dxy, az.om * xdy, az.dom * fxy, q.v[0]);
      add(az.o2 * dxy, az.o2 * xdy, az.do2 * fxy, q.v[3]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T tri = fxy * az.f[c];
        add(ax.dq * tri + B * dxy * az.f[c], ay.dq * tri + B * xdy * az.f[c], az.dq * tri + B * fxy * az.d[c],
            q.v[c + 1]);
      }
    }
  // x-outer columns (x layer 0: om, 3: o2), inner y and z layers
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const Quad<T> qm = load_quad<T>(quads + (size_t)(ix[0] + iy[b + 1] + iz) * 4);
    const Quad<T> qp = load_quad<T>(quads + (size_t)(ix[3] + iy[b + 1] + iz) * 4);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T yz = ay.f[b] * az.f[c], dyz = ay.d[b] * az.f[c], ydz = ay.f[b] * az.d[c];
      add(ax.dom * yz, ax.om * dyz, ax.om * ydz, qm.v[c + 1]);
      add(ax.do2 * yz, ax.o2 * dyz, ax.o2 * ydz, qp.v[c + 1]);
    }
  }
  // y-outer columns (y layer 0: om, 3: o2), inner x and z layers
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const Quad<T> qm = load_quad<T>(quads + (size_t)(ix[a + 1] + iy[0] + iz) * 4);
    const Quad<T> qp = load_quad<T>(quads + (size_t)(ix[a + 1] + iy[3] + iz) * 4);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T xz = ax.f[a] * az.f[c], dxz = ax.d[a] * az.f[c], xdz = ax.f[a] * az.d[c];
      add(ay.om * dxz, ay.dom * xz, ay.om * xdz, qm.v[c + 1]);
      add(ay.o2 * dxz, ay.do2 * xz, ay.o2 * xdz, qp.v[c + 1]);
    }
  }
  return A3<T>{s.x * w_inv_h, s.y * w_inv_h, s.z * w_inv_h};
}

// phibar (H^3) -> its z-quads (4 H^3): quad n = phibar at z - 1, z, z + 1, z + 2 (periodic).
template <typename T>
__global__ void __launch_bounds__(256) k_adj_quads(const T* __restrict__ phibar, T* __restrict__ quads, int H,
                                                   int64_t H3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < H3; i += (int64_t)gridDim.x * blockDim.x) {
    const int z = (int)(i & (H - 1));
    const int64_t row = i - z;
    T* q = quads + (size_t)i * 4;
    q[0] = phibar[row + ((z - 1) & (H - 1))];
    q[1] = phibar[i];
    q[2] = phibar[row + ((z + 1) & (H - 1))];
    q[3] = phibar[row + ((z + 2) & (H - 1))];
  }
}

// Add (a, b, c) to one (x, y, z, -) node of the interleaved cotangent grid:
// one 16-byte vector reduction in single precision (one L2 sector operation
// instead of three), three scalar ones in double precision.
template <typename T> __device__ __forceinline__ void red_node3(T* node, T a, T b, T c);
template <> __device__ __forceinline__ void red_node3<float>(float* node, float a, float b, float c) {
  atomicAdd(reinterpret_cast<float4*>(node), make_float4(a, b, c, 0.f));
}
template <> __device__ __forceinline__ void red_node3<double>(double* node, double a, double b, double c) {
  atomicAdd(node, a);
  atomicAdd(node + 1, b);
  atomicAdd(node + 2, c);
}

// One (x, y, z, -) node of the gradient grids, read through the read-only path.
template <typename T> struct Node4;
template <> struct Node4<float> {
  static __device__ __forceinline__ A3<float> load(const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z};
  }
};
template <> struct Node4<double> {
  static __device__ __forceinline__ A3<double> load(const double* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y, __ldg(p + 2)};
  }
};

// Xbar record of one particle: (x, y, z, 0).
template <typename T> struct Rec4;
template <> struct Rec4<float> {
  static __device__ __forceinline__ A3<float> load(const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z};
  }
  static __device__ __forceinline__ void store(float* p, float a, float b, float c) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, 0.f);
  }
};
template <> struct Rec4<double> {
  static __device__ __forceinline__ A3<double> load(const double* p) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    return {v.x, v.y, p[2]};
  }
  static __device__ __forceinline__ void store(double* p, double a, double b, double c) {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, 0.0);
  }
};

// Block sum of two values into FP64 accumulators (one atomic pair per block).
template <typename T> __device__ __forceinline__ void block_acc2(T a, T b, double* acc) {
  __shared__ double sa[32], sb[32];
  double da = (double)a, db = (double)b;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    da += __shfl_xor_sync(0xffffffffu, da, o);
    db += __shfl_xor_sync(0xffffffffu, db, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sa[wid] = da;
    sb[wid] = db;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    da = lane < nw ? sa[lane] : 0.0;
    db = lane < nw ? sb[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      da += __shfl_xor_sync(0xffffffffu, da, o);
      db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    if (lane == 0) {
      atomicAdd(acc, da);
      atomicAdd(acc + 1, db);
    }
  }
}

// One reverse step n for every particle.  In: X^{n-1} (entries in bin order
// with their ids, or in particle order), the gradient grids g^{n-1} as (gx,
// gy, gz, 0) nodes, phibar^{n-1} and Xbar^n; out: Xbar^{n-1} (in place), the
// gradient-grid cotangents gbar (H^3 interleaved (x, y, z, -) nodes,
// accumulated) and the sums for dJ/dchi and dJ/ds.
// G2P / P2G: the gather and deposit orders fixed at compile time (0: taken
// from the arguments at run time); the default pair (2, 4) compiles one
// stencil of each kind, which fits the kernel in 64 registers (four blocks
// per SM, no spills).
template <typename T, int G2P, int P2G>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? ((G2P && P2G) ? 4 : 2) : 1)
k_adj_step(AdjArgs<T> a) {
  const int g2p = G2P ? G2P : a.g2p, p2g = P2G ? P2G : a.p2g;
  T chi_part = T(0), s_part = T(0);
  const Geo<T> g = a.g;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.P; p += (int64_t)gridDim.x * blockDim.x) {
    const T x = a.x[p], y = a.y[p], z = a.z[p];
    const uint32_t id = a.id ? a.id[p] : (uint32_t)p;
    T* const rec = a.xb4 + (size_t)id * 4;
    const A3<T> b = Rec4<T>::load(rec);
    const T bx = b.x, by = b.y, bz = b.z;
    T nz[6];
    normals6(a.seed, (uint64_t)id, a.n, nz);
    // point where the drift gradient is gathered: X + W^- (half splitting) or X
    const T qx = a.split == 0 ? x + a.s_noise * nz[0] : x;
    const T qy = a.split == 0 ? y + a.s_noise * nz[1] : y;
    const T qz = a.split == 0 ? z + a.s_noise * nz[2] : z;
    // V = I* g (q) and its Jacobian J[d][e] = dV_d / dq_e
    T V[3] = {T(0), T(0), T(0)};
    T J[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
    stencil_grad_visit<T>(g2p, qx, qy, qz, g, [&](int idx, T f, T fx, T fy, T fz) {
      const A3<T> g3 = Node4<T>::load(a.grad4 + (size_t)idx * 4);   // one vector load per node
      const T v[3] = {g3.x, g3.y, g3.z};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        V[d] += f * v[d];
        J[d][0] += fx * v[d];
        J[d][1] += fy * v[d];
        J[d][2] += fz * v[d];
      }
    });
    chi_part += a.tau * (V[0] * bx + V[1] * by + V[2] * bz);
    const T ct = a.chitau * g.inv_h;   // J above is in lambda units: d/dq = (H/L) d/dlambda
    const T ybx = bx + ct * (J[0][0] * bx + J[1][0] * by + J[2][0] * bz);
    const T yby = by + ct * (J[0][1] * bx + J[1][1] * by + J[2][1] * bz);
    const T ybz = bz + ct * (J[0][2] * bx + J[1][2] * by + J[2][2] * bz);
    if (a.split == 0)
      s_part += nz[0] * ybx + nz[1] * yby + nz[2] * ybz + nz[3] * bx + nz[4] * by + nz[5] * bz;
    else
      s_part += nz[0] * bx + nz[1] * by + nz[2] * bz;
    // gbar_d += F_gamma(q) chi tau Xbar_d  (transpose of the gather)
    const T cbx = a.chitau * bx, cby = a.chitau * by, cbz = a.chitau * bz;
    stencil_grad_visit<T>(g2p, qx, qy, qz, g, [&](int idx, T f, T, T, T) {
      red_node3<T>(a.gbar + (size_t)idx * 4, f * cbx, f * cby, f * cbz);
    });
    // transpose of the deposit of X^{n-1}
    // (the Gamma_4 specialisation reads the z-quads; the run-time-order kernel phibar)
    const A3<T> dp = P2G == 4 ? deposit_adjoint4_quads<T>(a.phibar4, x, y, z, a.w_inv_h, g)
                              : deposit_adjoint<T>(a.phibar, p2g, x, y, z, a.w_inv_h, g);
    Rec4<T>::store(rec, ybx + dp.x, yby + dp.y, ybz + dp.z);
  }
  block_acc2<T>(chi_part, s_part, a.acc);
}

// Interleaved cotangent nodes -> three planes of H^3 (the transforms' input);
// the nodes are cleared for the next step's accumulation.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_planes(T* __restrict__ gbar4, T* __restrict__ planes, int64_t H3) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < H3; i += (int64_t)gridDim.x * blockDim.x) {
    T* node = gbar4 + (size_t)i * 4;
    planes[i] = node[0];
    planes[H3 + i] = node[1];
    planes[2 * H3 + i] = node[2];
    node[0] = T(0);
    node[1] = T(0);
    node[2] = T(0);
  }
}

// Terminal cotangent: Xbar^N = transpose of the deposit at X^N (particle
// order) applied to phibar^N.
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_terminal(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P,
               const T* __restrict__ phibar, int p2g, T w_inv_h, Geo<T> g, T* __restrict__ xb4) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const A3<T> dp = deposit_adjoint<T>(phibar, p2g, x[p], y[p], z[p], w_inv_h, g);
    Rec4<T>::store(xb4 + (size_t)p * 4, dp.x, dp.y, dp.z);
  }
}

// Fourier side of one reverse step on full 3D half spectra [H][H][H/2+1]:
//   abar <- A abar + sum_d conj(m_d) ghat_d,   m_d = 2 pi i q_d / L Phi_q (0 on q_d = -H/2),
//   betabar_next = L^-3 B abar  (written to `spec`, ready for the inverse transform
//   that gives the transpose of F_H).
template <typename T>
__global__ void __launch_bounds__(256)
k_adj_spectral(const cpx<T>* __restrict__ ghat, cpx<T>* __restrict__ abar, cpx<T>* __restrict__ spec, int H,
               SpecParams sp) {
  const int nh = H / 2 + 1;
  const size_t S = (size_t)H * H * nh;
  const T two_pi_L = T(6.283185307179586 / sp.L);
  const T filt = sp.H0 > 0 ? T(-2.0 * 9.869604401089358 / (sp.H0 * sp.H0)) : T(0);
  const T tau_eps = T(sp.tau / sp.eps), eps_tau = T(sp.eps / sp.tau), k2 = T(sp.k2), tau = T(sp.tau);
  const T inv_L3 = T(sp.inv_L3);
  // 32-bit index arithmetic (S < 2^31 for H <= 256; a 64-bit division costs
  // several times more than the element's own work)
  const unsigned S32 = (unsigned)S, unh = (unsigned)nh, uH = (unsigned)H;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < S32; i += gridDim.x * blockDim.x) {
    const unsigned row = i / unh;
    const int mz = (int)(i - row * unh);
    const int my = (int)(row % uH);
    const int mx = (int)(row / uH);
    const int qx = mx < H / 2 ? mx : mx - H;
    const int qy = my < H / 2 ? my : my - H;
    const int qz = mz < H / 2 ? mz : mz - H;
    const T q2 = T(qx * qx + qy * qy + qz * qz);
    const T lam = two_pi_L * two_pi_L * q2 + k2;
    T A, B;
    if (sp.propagator == 0) {
      A = T(1) / (T(1) + tau_eps * lam);
      B = T(1) / (lam + eps_tau);
    } else {
      A = t_exp(-tau_eps * lam);
      B = A * tau;
    }
    const T Phi = sp.H0 > 0 ? t_exp(filt * q2) : T(1);
    cpx<T> acc{T(0), T(0)};
    const int qd[3] = {qx, qy, qz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (qd[d] == -H / 2) continue;
      const T yd = two_pi_L * T(qd[d]) * Phi;
      const cpx<T> gh = ghat[d * S + i];
      // conj(i yd) (gh.x + i gh.y) = yd (gh.y - i gh.x)
      acc.x += yd * gh.y;
      acc.y -= yd * gh.x;
    }
    const cpx<T> ab = abar[i];
    const cpx<T> an{A * ab.x + acc.x, A * ab.y + acc.y};
    abar[i] = an;
    spec[i] = cpx<T>{inv_L3 * B * an.x, inv_L3 * B * an.y};
  }
}

int grid_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

}  // namespace

template <typename T> cudaError_t launch_adj_step(const AdjArgs<T>& a, cudaStream_t s) {
  if (a.P <= 0) return cudaSuccess;
  auto k = (a.g2p == 2 && a.p2g == 4) ? k_adj_step<T, 2, 4> : k_adj_step<T, 0, 0>;
  k<<<grid_blocks(a.P), 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_adj_quads(const T* phibar, T* quads, int H, cudaStream_t s) {
  const int64_t H3 = (int64_t)H * H * H;
  k_adj_quads<T><<<grid_blocks(H3), 256, 0, s>>>(phibar, quads, H, H3);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_adj_planes(T* gbar4, T* planes, int64_t H3, cudaStream_t s) {
  k_adj_planes<T><<<grid_blocks(H3), 256, 0, s>>>(gbar4, planes, H3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_terminal(const T* x, const T* y, const T* z, int64_t P, const T* phibar, int p2g, T w_inv_h,
                                Geo<T> g, T* xb4, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  k_adj_terminal<T><<<grid_blocks(P), 256, 0, s>>>(x, y, z, P, phibar, p2g, w_inv_h, g, xb4);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_spectral(const cpx<T>* ghat, cpx<T>* abar, cpx<T>* spec, int H, SpecParams sp,
                                cudaStream_t s) {
  const int64_t S = (int64_t)H * H * (H / 2 + 1);
  k_adj_spectral<T><<<grid_blocks(S), 256, 0, s>>>(ghat, abar, spec, H, sp);
  return cudaGetLastError();
}

#define SIPF_ADJ_INST(T)                                                                                          \
  template cudaError_t launch_adj_step<T>(const AdjArgs<T>&, cudaStream_t);                                      \
  template cudaError_t launch_adj_planes<T>(T*, T*, int64_t, cudaStream_t);                                      \
  template cudaError_t launch_adj_quads<T>(const T*, T*, int, cudaStream_t);                                     \
  template cudaError_t launch_adj_terminal<T>(const T*, const T*, const T*, int64_t, const T*, int, T, Geo<T>, T*, \
                                              cudaStream_t);                                                     \
  template cudaError_t launch_adj_spectral<T>(const cpx<T>*, cpx<T>*, cpx<T>*, int, SpecParams, cudaStream_t);
SIPF_ADJ_INST(float)
SIPF_ADJ_INST(double)
#undef SIPF_ADJ_INST

}  // namespace sipf
