// Two-dimensional SIPF-PIC: the parabolic-elliptic variant of Sec. 5.2
// (Keller-Segel with eps = 0 in 2D: the critical-mass and second-moment
// experiments), and the 2D parabolic-parabolic system for eps > 0.
//
// One step n on [-L/2, L/2)^2 with an H x H grid (H <= 256):
//   the forward F_H of the deposited masses (the 3D code's
//   row and column FFT kernels over an H x H array), the spectral kernel below
//   (eps = 0: alpha = beta / (|y|^2 + k^2), the field of level n-1 for the
//   drift; eps > 0: the implicit update of Eq. (alpha_hat_update) with the
//   drift from alpha^(n-1)), the two filtered gradient spectra, their inverse
//   transforms into (gx, gy, 0, 0) nodes, the move (first Philox block:
//   W^- = s (z0, z1), W^+ = s (z2, z3); bilinear gather; wrap), and the
//   deposit of X^n with the 12-node 2D analogue of Eq. (4ord) (or bilinear).
// Particles stay in particle order (no tile bins) and deposit with global
// reductions: the 2D grids (at most 256^2 nodes) live in L2.
#include <cuda_runtime.h>
#include <math.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/sipf.h"
#include "sipf_internal.h"

namespace sipf {
double filter_scale(const sipf_params& p);   // sipf_api.cu

namespace {

constexpr int kT2 = 256;

inline int grid_for2(int64_t n, int threads, int cap = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// The 2D stencils on the periodic H x H grid: fn(flat node index, w F).
// Order 4: inner nodes (a, b) in {0,1}^2 carry the bilinear weight times
// 1 + (lx (1 - lx) + ly (1 - ly)) / 2; the outer node with index -1 or 2 on
// one axis the cubic factor of that axis times the linear weight of the other.
template <typename T, typename Fn>
__device__ __forceinline__ void stencil2d(int order, int cx, int cy, T lx, T ly, T w, int H, int mask, Fn&& fn) {
  const int x0 = (cx & mask) * H, x1 = ((cx + 1) & mask) * H;
  const int y0 = cy & mask, y1 = (cy + 1) & mask;
  const T wx0 = (T(1) - lx) * w, wx1 = lx * w, wy0 = T(1) - ly, wy1 = ly;
  if (order == 2) {
    fn(x0 + y0, wx0 * wy0);
    fn(x0 + y1, wx0 * wy1);
    fn(x1 + y0, wx1 * wy0);
    fn(x1 + y1, wx1 * wy1);
    return;
  }
  const T boost = T(1) + T(0.5) * (lx * (T(1) - lx) + ly * (T(1) - ly));
  const T cxl = lx * (T(1) - lx) * T(1.0 / 6.0), cyl = ly * (T(1) - ly) * T(1.0 / 6.0);
  const T xm = -(T(2) - lx) * cxl * w, x2 = -(T(1) + lx) * cxl * w;   // indices -1, 2 on x (weight folded in)
  const T ym = -(T(2) - ly) * cyl, y2 = -(T(1) + ly) * cyl;           // indices -1, 2 on y
  const int xm_i = ((cx - 1) & mask) * H, x2_i = ((cx + 2) & mask) * H;
  const int ym_i = (cy - 1) & mask, y2_i = (cy + 2) & mask;
  fn(x0 + y0, wx0 * wy0 * boost);
  fn(x0 + y1, wx0 * wy1 * boost);
  fn(x1 + y0, wx1 * wy0 * boost);
  fn(x1 + y1, wx1 * wy1 * boost);
  fn(xm_i + y0, xm * wy0);
  fn(xm_i + y1, xm * wy1);
  fn(x2_i + y0, x2 * wy0);
  fn(x2_i + y1, x2 * wy1);
  fn(x0 + ym_i, wx0 * ym);
  fn(x1 + ym_i, wx1 * ym);
  fn(x0 + y2_i, wx0 * y2);
  fn(x1 + y2_i, wx1 * y2);
}

template <typename T>
__global__ void __launch_bounds__(kT2)
k2_deposit(const T* __restrict__ x, const T* __restrict__ y, int64_t P, Geo<T> g, T w, int order,
           T* __restrict__ phi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    int cx, cy;
    T lx, ly;
    cell_lambda(x[p], g, cx, lx);
    cell_lambda(y[p], g, cy, ly);
    stencil2d<T>(order, cx, cy, lx, ly, w, g.H, g.mask, [&](int idx, T f) { atomicAdd(phi + idx, f); });
  }
}

struct Spec2D {
  double L, inv_L2, tau, eps, k2, H0;
  int mode;   // 0: step (field + gradients), 1: density Phi beta into component 0
};

// One thread per mode of the H x (H/2+1) half spectrum.
template <typename T>
__global__ void __launch_bounds__(kT2)
k2_spectral(const cpx<T>* __restrict__ T1, cpx<T>* __restrict__ alpha, cpx<T>* __restrict__ T2, int H, Spec2D sp) {
  const int NH = H / 2 + 1;
  const int S = H * NH;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= S) return;
  const int kx = m / NH, ky = m - kx * NH;
  const int qx = kx < H / 2 ? kx : kx - H;
  const int qy = ky < H / 2 ? ky : ky - H;
  const T q2 = (T)(qx * qx + qy * qy);
  const T Phi = sp.H0 > 0 ? t_exp((T)(-2.0 * M_PI * M_PI / (sp.H0 * sp.H0)) * q2) : T(1);
  cpx<T> beta = T1[m];
  beta.x *= (T)sp.inv_L2;
  beta.y *= (T)sp.inv_L2;
  if (sp.mode == 1) {
    T2[m] = cpx<T>{beta.x * Phi, beta.y * Phi};
    return;
  }
  const T two_pi_L = (T)(2.0 * M_PI / sp.L);
  const T lam = two_pi_L * two_pi_L * q2 + (T)sp.k2;
  cpx<T> a;   // the field that drives this step's move
  if (sp.eps == 0.0) {
    a = lam > T(0) ? cpx<T>{beta.x / lam, beta.y / lam} : cpx<T>{T(0), T(0)};
    alpha[m] = a;
  } else {
    a = alpha[m];
    const T kappa = T(1) / (T(1) + (T)(sp.tau / sp.eps) * lam);
    const T src = T(1) / (lam + (T)(sp.eps / sp.tau));
    alpha[m] = cpx<T>{kappa * a.x + src * beta.x, kappa * a.y + src * beta.y};
  }
  const T yx = two_pi_L * (T)qx * Phi, yy = two_pi_L * (T)qy * Phi;
  T2[m] = qx != -H / 2 ? cpx<T>{-yx * a.y, yx * a.x} : cpx<T>{T(0), T(0)};
  T2[S + m] = qy != -H / 2 ? cpx<T>{-yy * a.y, yy * a.x} : cpx<T>{T(0), T(0)};
}

template <typename T>
__global__ void __launch_bounds__(kT2)
k2_move(T* __restrict__ x, T* __restrict__ y, int64_t P, Geo<T> g, const T* __restrict__ grad4, int g2p, int split,
        T s_noise, T chitau, uint64_t seed, uint32_t n, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    T z[4];
    normals4(seed, (uint64_t)p, n, z);
    T px = x[p], py = y[p];
    if (split == 0) {   // Z = X + W^- + chi tau I*(grad c)(X + W^-),  X^n = Z + W^+
      px += s_noise * z[0];
      py += s_noise * z[1];
    }
    int cx, cy;
    T lx, ly;
    cell_lambda(px, g, cx, lx);
    cell_lambda(py, g, cy, ly);
    T gx = T(0), gy = T(0);
    stencil2d<T>(g2p, cx, cy, lx, ly, T(1), g.H, g.mask, [&](int idx, T f) {
      gx += f * grad4[(size_t)idx * 4];
      gy += f * grad4[(size_t)idx * 4 + 1];
    });
    if (split == 0) {
      px = wrap_coord((px + chitau * gx) + s_noise * z[2], g);
      py = wrap_coord((py + chitau * gy) + s_noise * z[3], g);
    } else {            // X^n = X + chi tau I*(grad c)(X) + W,  W ~ N(0, 2 mu tau I)
      px = wrap_coord((px + chitau * gx) + s_noise * z[0], g);
      py = wrap_coord((py + chitau * gy) + s_noise * z[1], g);
    }
    if (!(t_finite(px) && t_finite(py))) atomicOr(err, 1);
    x[p] = px;
    y[p] = py;
  }
}

__device__ __forceinline__ double warp_sum2(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc[0] += sum |X|^2, acc[1] += sum of the grid (mass)
template <typename T>
__global__ void __launch_bounds__(kT2)
k2_sums(const T* __restrict__ x, const T* __restrict__ y, int64_t P, const T* __restrict__ phi, int64_t N,
        double* acc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double m2 = 0.0, mass = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride)
    m2 += (double)x[p] * x[p] + (double)y[p] * y[p];
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) mass += (double)phi[j];
  m2 = warp_sum2(m2);
  mass = warp_sum2(mass);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, m2);
    atomicAdd(acc + 1, mass);
  }
}

// acc[2] += energy of modes with ||q|| >= 4, acc[3] += total (full spectrum:
// the columns ky = 0 and ky = H/2 once, the others twice)
template <typename T>
__global__ void __launch_bounds__(kT2) k2_energy(const cpx<T>* __restrict__ alpha, int H, double* acc) {
  const int NH = H / 2 + 1, S = H * NH;
  double hi = 0.0, tot = 0.0;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < S; m += gridDim.x * blockDim.x) {
    const int kx = m / NH, ky = m - kx * NH;
    const int qx = kx < H / 2 ? kx : kx - H, qy = ky < H / 2 ? ky : ky - H;
    const double e = ((double)alpha[m].x * alpha[m].x + (double)alpha[m].y * alpha[m].y) *
                     ((ky == 0 || ky == H / 2) ? 1.0 : 2.0);
    tot += e;
    if (qx * qx + qy * qy >= 16) hi += e;
  }
  hi = warp_sum2(hi);
  tot = warp_sum2(tot);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 2, hi);
    atomicAdd(acc + 3, tot);
  }
}

template <typename T>
__global__ void __launch_bounds__(kT2)
k2_load_aos(const double* __restrict__ X, int64_t P, Geo<T> g, T* __restrict__ x, T* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    x[p] = wrap_coord((T)X[2 * p], g);
    y[p] = wrap_coord((T)X[2 * p + 1], g);
  }
}

template <typename T>
__global__ void __launch_bounds__(kT2)
k2_store_aos(const T* __restrict__ x, const T* __restrict__ y, int64_t P, double* __restrict__ X) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    X[2 * p] = (double)x[p];
    X[2 * p + 1] = (double)y[p];
  }
}

}  // namespace
}  // namespace sipf

using namespace sipf;

struct sipf2d_ctx {
  sipf_params p{};
  double H0 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0;
  size_t esz = 4;
  void* x = nullptr;       // positions, particle order
  void* y = nullptr;
  void* phi = nullptr;     // H^2 deposited masses
  void* T1 = nullptr;      // H x (H/2+1) complex: forward transform
  void* alpha = nullptr;   // field spectrum (eps = 0: of the last level used; eps > 0: alpha^(n))
  void* T2 = nullptr;      // 3 half spectra: the gradient spectra and a zero third
  void* grad = nullptr;    // H^2 nodes (gx, gy, 0, 0); also the density scratch
  double* acc = nullptr;   // FP64 sums: [0] sum |X|^2, [1] mass, [2] HF energy, [3] total energy, [4] max
  double* aos = nullptr;   // P x 2 staging of host positions
  int* err = nullptr;
  int64_t S() const { return (int64_t)p.H * (p.H / 2 + 1); }
  int64_t N() const { return (int64_t)p.H * p.H; }
};

namespace {

#define SIPF2_CK(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return report_cuda(e_, #call);      \
  } while (0)

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate2d(const sipf_params* p) {
  if (!p) return report_error(SIPF_EINVAL, "params is NULL");
  auto bad = [](const char* f) { return report_error(SIPF_EINVAL, std::string("invalid 2D parameter: ") + f); };
  if (!(p->P >= 1 && p->P <= (1LL << 30))) return bad("P (1 <= P <= 2^30)");
  if (!pow2(p->H) || p->H < 8 || p->H > 256) return bad("H (power of two in [8, 256])");
  if (p->precision != 32 && p->precision != 64) return bad("precision (32 or 64)");
  if (!(isfinite(p->L) && p->L > 0)) return bad("L (> 0)");
  if (!(isfinite(p->mass) && p->mass > 0)) return bad("mass (> 0)");
  if (!(isfinite(p->chi) && p->chi >= 0)) return bad("chi (>= 0)");
  if (!(isfinite(p->mu) && p->mu > 0)) return bad("mu (> 0)");
  if (!(isfinite(p->eps) && p->eps >= 0)) return bad("eps (>= 0; 0 is the parabolic-elliptic system)");
  if (!(isfinite(p->k) && p->k >= 0)) return bad("k (>= 0)");
  if (!(isfinite(p->dt) && p->dt > 0)) return bad("dt (> 0)");
  if (!isfinite(p->H0)) return bad("H0 (finite)");
  if (p->p2g_order != 2 && p->p2g_order != 4) return bad("p2g_order (2 or 4)");
  if (p->g2p_order != 2 && p->g2p_order != 4) return bad("g2p_order (2 or 4)");
  if (p->splitting != SIPF_SPLIT_HALF && p->splitting != SIPF_SPLIT_PLAIN) return bad("splitting");
  if (p->deposit_mode != SIPF_DEPOSIT_ATOMIC) return bad("deposit_mode (atomic only in 2D)");
  if (p->propagator != SIPF_PROP_IMPLICIT) return bad("propagator (implicit only in 2D)");
  return SIPF_OK;
}

void free2d(sipf2d_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* q : {c->x, c->y, c->phi, c->T1, c->alpha, c->T2, c->grad, (void*)c->acc, (void*)c->aos, (void*)c->err})
    cudaFree(q);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

template <typename T> Geo<T> geo2(const sipf2d_ctx* c) { return make_geo<T>(c->p.L, c->p.H); }

template <typename T> int deposit2(sipf2d_ctx* c) {
  const T w = (T)(c->p.mass / (double)c->p.P);
  k2_deposit<T><<<grid_for2(c->p.P, kT2), kT2, 0, c->stream>>>((const T*)c->x, (const T*)c->y, c->p.P, geo2<T>(c), w,
                                                                c->p.p2g_order, (T*)c->phi);
  SIPF2_CK(cudaGetLastError());
  return SIPF_OK;
}

Spec2D spec2(const sipf2d_ctx* c, int mode) {
  Spec2D s;
  s.L = c->p.L;
  s.inv_L2 = 1.0 / (c->p.L * c->p.L);
  s.tau = c->p.dt;
  s.eps = c->p.eps;
  s.k2 = c->p.k * c->p.k;
  s.H0 = c->H0;
  s.mode = mode;
  return s;
}

// F_H of phi (cleared as it is read if `clear`) into T1.
template <typename T> int forward2(sipf2d_ctx* c, bool clear, double* mass_acc) {
  const int H = c->p.H;
  SIPF2_CK(launch_rows_r2c<T>(c->phi, 0, 1.0, clear, (cpx<T>*)c->T1, H, H, mass_acc, c->stream));
  SIPF2_CK(launch_cols<T>((cpx<T>*)c->T1, H, 1, H / 2 + 1, 1, 0, -1, 1.0, c->stream));
  return SIPF_OK;
}

template <typename T> int step2(sipf2d_ctx* c, int64_t nsteps) {
  const int H = c->p.H;
  const size_t S = (size_t)c->S();
  const T s_noise = (T)(c->p.splitting == SIPF_SPLIT_HALF ? sqrt(c->p.mu * c->p.dt) : sqrt(2.0 * c->p.mu * c->p.dt));
  for (int64_t i = 0; i < nsteps; ++i) {
    int r = forward2<T>(c, true, nullptr);
    if (r) return r;
    k2_spectral<T><<<(unsigned)((S + kT2 - 1) / kT2), kT2, 0, c->stream>>>(
        (const cpx<T>*)c->T1, (cpx<T>*)c->alpha, (cpx<T>*)c->T2, H, spec2(c, 0));
    SIPF2_CK(cudaGetLastError());
    SIPF2_CK(launch_cols<T>((cpx<T>*)c->T2, H, 1, H / 2 + 1, 2, S, +1, 1.0, c->stream));
    SIPF2_CK(launch_rows_c2r<T>((const cpx<T>*)c->T2, 3, S, (T*)c->grad, H, H, nullptr, c->stream));
    k2_move<T><<<grid_for2(c->p.P, kT2), kT2, 0, c->stream>>>(
        (T*)c->x, (T*)c->y, c->p.P, geo2<T>(c), (const T*)c->grad, c->p.g2p_order, c->p.splitting, s_noise,
        (T)(c->p.chi * c->p.dt), c->p.seed, (uint32_t)(c->n + 1), c->err);
    SIPF2_CK(cudaGetLastError());
    c->n += 1;
    r = deposit2<T>(c);
    if (r) return r;
  }
  return SIPF_OK;
}

template <typename T> int init_positions2(sipf2d_ctx* c, const double* X0) {
  const size_t bytes = (size_t)c->p.P * 2 * sizeof(double);
  SIPF2_CK(cudaMemcpyAsync(c->aos, X0, bytes, cudaMemcpyHostToDevice, c->stream));
  k2_load_aos<T><<<grid_for2(c->p.P, kT2), kT2, 0, c->stream>>>(c->aos, c->p.P, geo2<T>(c), (T*)c->x, (T*)c->y);
  SIPF2_CK(cudaGetLastError());
  SIPF2_CK(cudaMemsetAsync(c->phi, 0, (size_t)c->N() * c->esz, c->stream));
  return deposit2<T>(c);
}

template <typename T> int positions2(sipf2d_ctx* c, double* out) {
  k2_store_aos<T><<<grid_for2(c->p.P, kT2), kT2, 0, c->stream>>>((const T*)c->x, (const T*)c->y, c->p.P, c->aos);
  SIPF2_CK(cudaGetLastError());
  SIPF2_CK(cudaMemcpyAsync(out, c->aos, (size_t)c->p.P * 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  SIPF2_CK(cudaStreamSynchronize(c->stream));
  return SIPF_OK;
}

template <typename T> int copy_to_host2(sipf2d_ctx* c, const void* src, size_t n, double* out, double scale) {
  std::vector<T> h(n);
  SIPF2_CK(cudaMemcpyAsync(h.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  SIPF2_CK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < n; ++i) out[i] = (double)h[i] * scale;
  return SIPF_OK;
}

// rho_num = F_H^-1(Phi F_H I rho-hat) (filtered) into grad, max into acc[4]
template <typename T> int density_num2(sipf2d_ctx* c, int filtered) {
  const int H = c->p.H;
  const size_t S = (size_t)c->S();
  int r = forward2<T>(c, false, nullptr);
  if (r) return r;
  Spec2D sp = spec2(c, 1);
  if (!filtered) sp.H0 = 0.0;
  k2_spectral<T><<<(unsigned)((S + kT2 - 1) / kT2), kT2, 0, c->stream>>>(
      (const cpx<T>*)c->T1, (cpx<T>*)c->alpha, (cpx<T>*)c->T2, H, sp);
  SIPF2_CK(cudaGetLastError());
  SIPF2_CK(launch_cols<T>((cpx<T>*)c->T2, H, 1, H / 2 + 1, 1, 0, +1, 1.0, c->stream));
  // (only the first spectrum is used; the third, read as zeros by the step's
  // node writer, is never written)
  SIPF2_CK(launch_rows_c2r<T>((const cpx<T>*)c->T2, 1, 0, (T*)c->grad, H, H, c->acc + 4, c->stream));
  return SIPF_OK;
}

template <typename T> int diag2(sipf2d_ctx* c, sipf_diag* d) {
  // acc[4] holds the maximum as an order-preserving 64-bit integer key
  double init[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  {
    const double ninf = -INFINITY;
    long long b;
    memcpy(&b, &ninf, 8);
    b ^= 0x7fffffffffffffffLL;
    memcpy(&init[4], &b, 8);
  }
  SIPF2_CK(cudaMemcpyAsync(c->acc, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
  k2_sums<T><<<grid_for2(c->p.P > c->N() ? c->p.P : c->N(), kT2, 152 * 8), kT2, 0, c->stream>>>(
      (const T*)c->x, (const T*)c->y, c->p.P, (const T*)c->phi, c->N(), c->acc);
  SIPF2_CK(cudaGetLastError());
  k2_energy<T><<<grid_for2(c->S(), kT2, 152 * 8), kT2, 0, c->stream>>>((const cpx<T>*)c->alpha, c->p.H, c->acc);
  SIPF2_CK(cudaGetLastError());
  int r = density_num2<T>(c, c->H0 > 0 ? 1 : 0);
  if (r) return r;
  double h[5];
  SIPF2_CK(cudaMemcpyAsync(h, c->acc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  SIPF2_CK(cudaStreamSynchronize(c->stream));
  memset(d, 0, sizeof(*d));
  d->m2 = h[0] / (double)c->p.P;
  d->mass = h[1];
  d->hf_frac = h[3] > 0 ? h[2] / h[3] : 0.0;
  long long b;
  memcpy(&b, &h[4], 8);
  if (b < 0) b ^= 0x7fffffffffffffffLL;
  memcpy(&d->peak, &b, 8);
  d->step = c->n;
  return SIPF_OK;
}

#define DISPATCH2(c, fn, ...) ((c)->p.precision == 64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

}  // namespace

extern "C" {

int sipf2d_init(const sipf_params* p, const double* X0, void* stream, sipf2d_ctx** out) {
  if (!out) return report_error(SIPF_EINVAL, "out is NULL");
  *out = nullptr;
  int r = validate2d(p);
  if (r) return r;
  if (!X0) return report_error(SIPF_EINVAL, "X0 is NULL");
  for (int64_t i = 0; i < 2 * p->P; ++i)
    if (!isfinite(X0[i])) return report_error(SIPF_ENONFINITE, "X0 holds a non-finite coordinate");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return report_error(SIPF_ENODEV, "no CUDA device");
  cudaError_t e = ensure_device_tables();
  if (e != cudaSuccess) return report_cuda(e, "ensure_device_tables");
  sipf2d_ctx* c = new sipf2d_ctx();
  c->p = *p;
  c->H0 = filter_scale(*p);
  c->esz = p->precision == 64 ? 8 : 4;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return report_cuda(e, "cudaStreamCreate");
    }
    c->own_stream = true;
  }
  const size_t P = (size_t)p->P, N = (size_t)c->N(), S = (size_t)c->S();
  e = cudaMalloc(&c->x, P * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->y, P * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->phi, N * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->T1, S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->alpha, S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->T2, 3 * S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->grad, 4 * N * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->acc, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->aos, P * 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->alpha, 0, S * 2 * c->esz, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->T2, 0, 3 * S * 2 * c->esz, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) {
    free2d(c);
    return report_cuda(e, "sipf2d_init allocation");
  }
  r = DISPATCH2(c, init_positions2, c, X0);
  if (r) {
    free2d(c);
    return r;
  }
  *out = c;
  return SIPF_OK;
}

int sipf2d_step(sipf2d_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return report_error(SIPF_EINVAL, "sipf2d_step arguments");
  return DISPATCH2(c, step2, c, nsteps);
}

int64_t sipf2d_current_step(const sipf2d_ctx* c) { return c ? c->n : -1; }

int sipf2d_positions(sipf2d_ctx* c, double* out) {
  if (!c || !out) return report_error(SIPF_EINVAL, "NULL argument");
  return DISPATCH2(c, positions2, c, out);
}

int sipf2d_spectrum(sipf2d_ctx* c, double* out) {
  if (!c || !out) return report_error(SIPF_EINVAL, "NULL argument");
  return DISPATCH2(c, copy_to_host2, c, c->alpha, (size_t)c->S() * 2, out, 1.0);
}

int sipf2d_density(sipf2d_ctx* c, double* out, int filtered) {
  if (!c || !out) return report_error(SIPF_EINVAL, "NULL argument");
  const double h2 = (c->p.L / c->p.H) * (c->p.L / c->p.H);
  if (!filtered) return DISPATCH2(c, copy_to_host2, c, c->phi, (size_t)c->N(), out, 1.0 / h2);
  int r = DISPATCH2(c, density_num2, c, 1);
  if (r) return r;
  return DISPATCH2(c, copy_to_host2, c, c->grad, (size_t)c->N(), out, 1.0);
}

int sipf2d_diagnostics(sipf2d_ctx* c, sipf_diag* out) {
  if (!c || !out) return report_error(SIPF_EINVAL, "NULL argument");
  return DISPATCH2(c, diag2, c, out);
}

int sipf2d_sync(sipf2d_ctx* c) {
  if (!c) return report_error(SIPF_EINVAL, "NULL context");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return report_cuda(e, "sipf2d_sync");
  int h = 0;
  e = cudaMemcpy(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return report_cuda(e, "sipf2d_sync");
  if (h & 1) return report_error(SIPF_ENONFINITE, "a position became non-finite");
  return SIPF_OK;
}

void sipf2d_destroy(sipf2d_ctx* c) { free2d(c); }

}  // extern "C"
