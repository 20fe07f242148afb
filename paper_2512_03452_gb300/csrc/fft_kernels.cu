// FFTs of the SIPF-PIC field solve (Sec. 3.2, Algorithm 4) on H^3 grids, H a
// power of two in [8, 256], float or double.
//
// Forward F_H: rows r2c along the fastest axis (two real rows per complex
// FFT), then c2c along the middle axis, then the x-axis pass fused with the
// implicit spectral update and the filtered gradient; the inverse runs the
// x axis back inside that same kernel, then the middle axis, then c2r rows.
// For H >= 32 each pencil of H = 32 E points is transformed by one warp
// (E values per lane: a radix-2 DFT in registers, then five shuffle stages);
// for H <= 128 the two inner axes of an x-plane are done in one block with
// the plane in shared memory (plane kernels kwp_*), for H = 256 by separate
// pencil passes (kwb_*).  H < 32 uses block-wide shared-memory transforms
// (k_*).  Every kernel's complex products spell out their roundings, so all
// shapes and paths give the same bits.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "sipf_internal.h"

namespace sipf {

// e^{-2 pi i m / 256}, m < 256, per device (written once by ensure_device_tables).
__device__ double2 g_twiddle[kNmax];

cudaError_t ensure_device_tables() {
  static std::mutex mu;
  static std::vector<bool> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, false);
  if (done[dev]) return cudaSuccess;
  double2 h[kNmax];
  for (int m = 0; m < kNmax; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)kNmax;
    h[m] = make_double2(cos(a), sin(a));
  }
  e = cudaMemcpyToSymbol(g_twiddle, h, sizeof(h));
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

__device__ __forceinline__ int brev(int j, int lg) { return (int)(__brev((unsigned)j) >> (32 - lg)); }

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* tw) {
  for (int i = threadIdx.x; i < kNmax / 2; i += blockDim.x) tw[i] = cpx<T>{(T)g_twiddle[i].x, (T)g_twiddle[i].y};
}

// In-place radix-2 DIT transform of `ncol` pencils of length n = 2^lgn in
// shared memory; element (j, c) at buf[j*ldj + c*ldc].  Input in bit-reversed
// order, output in natural order.  DIR = -1: e^{-i...} (forward), +1: inverse
// (unnormalised).  COLFAST: consecutive threads walk the pencil index c (use
// when ldc == 1), else the butterfly index.  ncol must be a power of two.
template <typename T, int DIR, bool COLFAST>
__device__ void smem_fft(cpx<T>* buf, const cpx<T>* tw, int lgn, int lgc, int ldj, int ldc) {
  const int n = 1 << lgn;
  const int nbf = (n >> 1) << lgc;
  for (int s = 0; s < lgn; ++s) {
    const int half = 1 << s;
    const int tws = (kNmax / 2) >> s;
    for (int t = threadIdx.x; t < nbf; t += blockDim.x) {
      int b, c;
      if (COLFAST) {
        c = t & ((1 << lgc) - 1);
        b = t >> lgc;
      } else {
        b = t & ((n >> 1) - 1);
        c = t >> (lgn - 1);
      }
      const int k = b & (half - 1);
      const int i0 = ((b >> s) << (s + 1)) + k;
      cpx<T> w = tw[k * tws];
      if (DIR > 0) w.y = -w.y;
      cpx<T>* p0 = buf + i0 * ldj + c * ldc;
      cpx<T>* p1 = p0 + half * ldj;
      const cpx<T> a = *p0;
      const cpx<T> v = cmul(*p1, w);
      *p0 = cadd(a, v);
      *p1 = csub(a, v);
    }
    __syncthreads();
  }
}

static inline int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// ---------------------------------------------------------------------------
// Rows r2c: rows 2c and 2c+1 of the block form z = a + i b; after the FFT,
// A_k = (Z_k + conj Z_{n-k})/2 and B_k = -i (Z_k - conj Z_{n-k})/2.
// ---------------------------------------------------------------------------
template <typename T, typename Tin>
__global__ void __launch_bounds__(kThreads)
k_rows_r2c(Tin* __restrict__ in, double in_scale, int zero_input, cpx<T>* __restrict__ out,
           int lgH, int rows, int RP, double* mass_acc) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* buf = tw + kNmax / 2;
  const int H = 1 << lgH, nh = H / 2 + 1, ld = H + 1;
  const int lgc = ilog2_dev(RP);
  load_twiddles(tw);
  const int row0 = blockIdx.x * 2 * RP;
  const int nrow = min(2 * RP, rows - row0);
  double msum = 0.0;
  for (int t = threadIdx.x; t < 2 * RP * H; t += blockDim.x) {
    const int r = t >> lgH, j = t & (H - 1);
    T v = T(0);
    if (r < nrow) {
      const size_t gi = (size_t)(row0 + r) * H + j;
      if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value) {
        v = (T)((double)(long long)in[gi] * in_scale);
      } else {
        v = (T)in[gi];
      }
      if (zero_input) in[gi] = Tin(0);
      msum += (double)v;
    }
    cpx<T>& e = buf[(r >> 1) * ld + brev(j, lgH)];
    if (r & 1) e.y = v; else e.x = v;
  }
  __syncthreads();
  smem_fft<T, -1, false>(buf, tw, lgH, lgc, 1, ld);
  for (int t = threadIdx.x; t < RP * nh; t += blockDim.x) {
    const int c = t / nh, k = t - c * nh;
    if (2 * c >= nrow) continue;
    const cpx<T> zk = buf[c * ld + k];
    const cpx<T> zm = cconj(buf[c * ld + ((H - k) & (H - 1))]);
    const cpx<T> A{(zk.x + zm.x) * T(0.5), (zk.y + zm.y) * T(0.5)};
    const cpx<T> d = csub(zk, zm);
    const cpx<T> B{d.y * T(0.5), -d.x * T(0.5)};
    out[(size_t)(row0 + 2 * c) * nh + k] = A;
    out[(size_t)(row0 + 2 * c + 1) * nh + k] = B;
  }
  if (mass_acc) {
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(mass_acc, msum);
  }
}

// ---------------------------------------------------------------------------
// c2c along the middle axis of [A][H][B]: block = (column chunk, a, component).
// ---------------------------------------------------------------------------
template <typename T, int DIR>
__global__ void __launch_bounds__(kThreads)
k_cols(cpx<T>* __restrict__ data, int lgH, int B, int lgBC, size_t comp_stride, T scale) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* buf = tw + kNmax / 2;
  const int H = 1 << lgH, BC = 1 << lgBC;
  load_twiddles(tw);
  cpx<T>* base = data + blockIdx.z * comp_stride + (size_t)blockIdx.y * H * B;
  const int b0 = blockIdx.x * BC;
  const int nb = min(BC, B - b0);
  for (int t = threadIdx.x; t < H * BC; t += blockDim.x) {
    const int j = t >> lgBC, c = t & (BC - 1);
    cpx<T> v{T(0), T(0)};
    if (c < nb) v = base[(size_t)j * B + b0 + c];
    buf[brev(j, lgH) * BC + c] = v;
  }
  __syncthreads();
  smem_fft<T, DIR, true>(buf, tw, lgH, lgBC, BC, 1);
  for (int t = threadIdx.x; t < H * BC; t += blockDim.x) {
    const int j = t >> lgBC, c = t & (BC - 1);
    if (c < nb) {
      cpx<T> v = buf[j * BC + c];
      base[(size_t)j * B + b0 + c] = cpx<T>{v.x * scale, v.y * scale};
    }
  }
}

// ---------------------------------------------------------------------------
// x-axis pass fused with the spectral work.  Columns m = ky*(H/2+1) + kz of the
// flattened (ky, kz) plane, all kx.  Slots of the shared buffer: 0 = beta,
// 1..3 = the outputs (inverse-transformed along x before they are stored).
//   kModeStep:     alpha^n = kappa alpha^{n-1} + src beta^{n-1}  (Eq. (alpha_hat_update)
//                  or the exponential propagator of Sec. 3.4) and
//                  G_d = i (2 pi q_d / L) Phi_q alpha^{n-1}, zero where q_d = -H/2.
//   kModeGradOnly: only G_d (alpha read, not updated; T1 unused).
//   kModeDensity:  G_0 = Phi_q beta_q  (rho_num, Sec. 5.2).
//   kModeField:    G_0 = alpha_q.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads)
k_spectral_x(const cpx<T>* __restrict__ T1, cpx<T>* __restrict__ alpha, cpx<T>* __restrict__ T2,
             int lgH, int lgBC, SpecParams sp, double* alpha0_shadow) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* buf = tw + kNmax / 2;
  const int H = 1 << lgH, BC = 1 << lgBC, nh = H / 2 + 1;
  const int B = H * nh;
  const size_t S = (size_t)H * B;
  const int ld = 4 * BC;
  load_twiddles(tw);
  const int b0 = blockIdx.x * BC;
  const int nb = min(BC, B - b0);
  constexpr bool needs_beta = (MODE == kModeStep || MODE == kModeDensity);
  if (needs_beta) {
    for (int t = threadIdx.x; t < H * BC; t += blockDim.x) {
      const int j = t >> lgBC, c = t & (BC - 1);
      cpx<T> v{T(0), T(0)};
      if (c < nb) v = T1[(size_t)j * B + b0 + c];
      buf[brev(j, lgH) * ld + c] = v;
    }
    __syncthreads();
    smem_fft<T, -1, true>(buf, tw, lgH, lgBC, ld, 1);
  }
  const T two_pi_L = (T)(2.0 * M_PI / sp.L);
  const T inv_L3 = (T)sp.inv_L3;
  const T tau_eps = (T)(sp.tau / sp.eps), eps_tau = (T)(sp.eps / sp.tau), k2 = (T)sp.k2, tau = (T)sp.tau;
  const T filt = sp.H0 > 0 ? (T)(-2.0 * M_PI * M_PI / (sp.H0 * sp.H0)) : T(0);
  for (int t = threadIdx.x; t < H * BC; t += blockDim.x) {
    const int j = t >> lgBC, c = t & (BC - 1);
    const int m = b0 + c;
    const int jr = brev(j, lgH);
    cpx<T> o1{T(0), T(0)}, o2{T(0), T(0)}, o3{T(0), T(0)};
    if (c < nb) {
      const int ky = m / nh, kz = m - ky * nh;
      const int qx = j < H / 2 ? j : j - H;
      const int qy = ky < H / 2 ? ky : ky - H;
      const int qz = kz < H / 2 ? kz : kz - H;
      const T q2 = (T)(qx * qx + qy * qy + qz * qz);
      const T Phi = sp.H0 > 0 ? t_exp(filt * q2) : T(1);
      const size_t gi = (size_t)j * B + m;
      if (MODE == kModeStep || MODE == kModeGradOnly) {
        const cpx<T> a = alpha[gi];
        if (MODE == kModeStep) {
          cpx<T> beta = buf[j * ld + c];
          beta.x *= inv_L3;
          beta.y *= inv_L3;
          const T lam = two_pi_L * two_pi_L * q2 + k2;
          cpx<T> an;
          if (sp.propagator == 0) {
            const T kappa = T(1) / (T(1) + tau_eps * lam);
            const T src = T(1) / (lam + eps_tau);
            an = cpx<T>{kappa * a.x + src * beta.x, kappa * a.y + src * beta.y};
          } else {
            const T kappa = t_exp(-tau_eps * lam);
            an = cpx<T>{kappa * (a.x + tau * beta.x), kappa * (a.y + tau * beta.y)};
          }
          alpha[gi] = an;
          if (m == 0 && j == 0 && alpha0_shadow) {
            const double lam0 = sp.k2;
            double s = *alpha0_shadow;
            if (sp.propagator == 0) s = s / (1.0 + sp.tau / sp.eps * lam0) + sp.beta0 / (lam0 + sp.eps / sp.tau);
            else s = exp(-sp.tau / sp.eps * lam0) * (s + sp.tau * sp.beta0);
            *alpha0_shadow = s;
          }
        }
        const T yx = two_pi_L * (T)qx * Phi, yy = two_pi_L * (T)qy * Phi, yz = two_pi_L * (T)qz * Phi;
        // i y a = (-y a.y, y a.x)
        if (qx != -H / 2) o1 = cpx<T>{-yx * a.y, yx * a.x};
        if (qy != -H / 2) o2 = cpx<T>{-yy * a.y, yy * a.x};
        if (qz != -H / 2) o3 = cpx<T>{-yz * a.y, yz * a.x};
      } else if (MODE == kModeDensity) {
        const cpx<T> beta = buf[j * ld + c];
        o1 = cpx<T>{beta.x * inv_L3 * Phi, beta.y * inv_L3 * Phi};
      } else {
        o1 = alpha[gi];
      }
    }
    buf[jr * ld + BC + c] = o1;
    buf[jr * ld + 2 * BC + c] = o2;
    buf[jr * ld + 3 * BC + c] = o3;
  }
  __syncthreads();
  constexpr int nout = (MODE == kModeStep || MODE == kModeGradOnly) ? 3 : 1;
  // inverse transform of slots 1..3 (slot 0 rides along as a fourth pencil)
  smem_fft<T, +1, true>(buf, tw, lgH, lgBC + 2, ld, 1);
  for (int t = threadIdx.x; t < H * BC; t += blockDim.x) {
    const int j = t >> lgBC, c = t & (BC - 1);
    if (c < nb) {
#pragma unroll
      for (int d = 0; d < nout; ++d) T2[d * S + (size_t)j * B + b0 + c] = buf[j * ld + (d + 1) * BC + c];
    }
  }
}

// ---------------------------------------------------------------------------
// Rows c2r: rows 2c, 2c+1 (Hermitian half spectra A, B) form Z = A + i B over
// the full index range (Z_{n-k} = conj A_k + i conj B_k); the inverse FFT
// gives a + i b.  The imaginary parts of the k = 0 and k = n/2 entries are
// dropped (they carry no real signal).
// ---------------------------------------------------------------------------
template <typename T, int NCOMP>
__global__ void __launch_bounds__(kThreads)
k_rows_c2r(const cpx<T>* __restrict__ in, size_t comp_stride, T* __restrict__ out, int lgH, int rows,
           int RP, double* max_acc) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* buf = tw + kNmax / 2;
  const int H = 1 << lgH, nh = H / 2 + 1, ld = H + 1;
  constexpr int NOUT = NCOMP == 3 ? 4 : 1;
  T* obuf = reinterpret_cast<T*>(buf + RP * ld);
  const int lgc = ilog2_dev(RP);
  load_twiddles(tw);
  const int row0 = blockIdx.x * 2 * RP;
  const int nrow = min(2 * RP, rows - row0);
  for (int d = 0; d < NCOMP; ++d) {
    const cpx<T>* src = in + d * comp_stride;
    for (int t = threadIdx.x; t < RP * H; t += blockDim.x) {
      const int c = t >> lgH, k = t & (H - 1);
      cpx<T> z{T(0), T(0)};
      if (2 * c < nrow) {
        const size_t ra = (size_t)(row0 + 2 * c) * nh, rb = ra + nh;
        cpx<T> A, Bv;
        if (k <= H / 2) {
          A = src[ra + k];
          Bv = src[rb + k];
          if (k == 0 || k == H / 2) { A.y = T(0); Bv.y = T(0); }
        } else {
          A = cconj(src[ra + (H - k)]);
          Bv = cconj(src[rb + (H - k)]);
        }
        z = cpx<T>{A.x - Bv.y, A.y + Bv.x};
      }
      buf[c * ld + brev(k, lgH)] = z;
    }
    __syncthreads();
    smem_fft<T, +1, false>(buf, tw, lgH, lgc, 1, ld);
    for (int t = threadIdx.x; t < 2 * RP * H; t += blockDim.x) {
      const int r = t >> lgH, j = t & (H - 1);
      const cpx<T> v = buf[(r >> 1) * ld + j];
      obuf[(r * H + j) * NOUT + d] = (r & 1) ? v.y : v.x;
    }
    __syncthreads();
  }
  double mx = -INFINITY;
  if (NOUT == 4) {
    for (int t = threadIdx.x; t < 2 * RP * H; t += blockDim.x) {
      const int r = t >> lgH;
      if (r < nrow) {
        const int j = t & (H - 1);
        T* o = out + ((size_t)(row0 + r) * H + j) * 4;
        const T* s = obuf + (r * H + j) * 4;
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(o) = make_float4(s[0], s[1], s[2], 0.f);
        } else {
          reinterpret_cast<double2*>(o)[0] = make_double2(s[0], s[1]);
          reinterpret_cast<double2*>(o)[1] = make_double2(s[2], 0.0);
        }
      }
    }
  } else {
    for (int t = threadIdx.x; t < 2 * RP * H; t += blockDim.x) {
      const int r = t >> lgH;
      if (r < nrow) {
        const T v = obuf[t];
        out[(size_t)row0 * H + t] = v;
        mx = fmax(mx, (double)v);
      }
    }
    if (max_acc) {
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0) {
        // order-preserving map of doubles onto signed 64-bit integers
        long long b = __double_as_longlong(mx);
        if (b < 0) b ^= 0x7fffffffffffffffLL;
        atomicMax(reinterpret_cast<long long*>(max_acc), b);
      }
    }
  }
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes);

// ===========================================================================
// Warp FFTs for H = 32 E, E in {2, 4, 8}.  A warp holds one pencil of
// length N = 32 E: lane l keeps elements j = l + 32 m (m < E) in registers.
//   1. E-point DFTs over m in registers (radix-2, twiddles from the table);
//   2. twiddle W_N^(l k1);
//   3. for each k1, a 32-point decimation-in-frequency across the lanes with
//      shfl_xor (no shared memory, no block barrier).
// Afterwards lane l, register k1 holds X[k1 + E bitrev5(l)].
// ===========================================================================
template <typename T, int DIR>
__device__ __forceinline__ cpx<T> twid(const cpx<T>* tw, int m) {
  cpx<T> w = tw[m & (kNmax - 1)];          // e^{-2 pi i m/256}
  if (DIR > 0) w.y = -w.y;
  return w;
}

// The warp kernels' shared twiddles: the full table (kNmax entries), then the
// per-lane twiddles of the warp FFT laid out lane-contiguously so a warp's
// reads hit distinct banks (read from the full table they are strided and
// collide up to 8-fold):
//   [kNmax + s + j]        cross-lane stage s (1..16), j = lane mod s: e^{-i pi j/s}
//   [kNmax + 32 k1 + lane] register twiddle W_N^(lane k1), k1 = 1..E-1
// Same values as the full table's entries, so the same bits.
constexpr int kTwLen = kNmax + 32 * 8;
template <typename T, int DIR> __device__ __forceinline__ cpx<T> twx(const cpx<T>* tw, int i) {
  cpx<T> w = tw[kNmax + i];
  if (DIR > 0) w.y = -w.y;
  return w;
}

template <typename T, int E, int DIR>
__device__ __forceinline__ void reg_dft(cpx<T> (&v)[E], const cpx<T>* tw) {
  if (E == 1) return;
  // bit-reverse the register order, then radix-2 decimation in time
  constexpr int LG = E == 2 ? 1 : (E == 4 ? 2 : 3);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < LG; ++b) r |= ((i >> b) & 1) << (LG - 1 - b);
    if (r > i) {
      const cpx<T> t = v[i];
      v[i] = v[r];
      v[r] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < E; half <<= 1) {
#pragma unroll
    for (int g = 0; g < E; g += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const cpx<T> w = twid<T, DIR>(tw, k * (kNmax / (2 * half)));
        const cpx<T> a = v[g + k];
        const cpx<T> b = cmul(v[g + k + half], w);
        v[g + k] = cadd(a, b);
        v[g + k + half] = csub(a, b);
      }
    }
  }
}

template <typename T> __device__ __forceinline__ cpx<T> shfl_xor_c(cpx<T> v, int s) {
  return cpx<T>{__shfl_xor_sync(0xFFFFFFFFu, v.x, s), __shfl_xor_sync(0xFFFFFFFFu, v.y, s)};
}

template <typename T, int E, int DIR>
__device__ __forceinline__ void warp_fft(cpx<T> (&v)[E], int lane, const cpx<T>* tw) {
  reg_dft<T, E, DIR>(v, tw);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], twx<T, DIR>(tw, 32 * k1 + lane));   // W_N^(lane k1)
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
    const cpx<T> w = up ? twx<T, DIR>(tw, s + (lane & (s - 1))) : cpx<T>{T(1), T(0)};
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      const cpx<T> u = shfl_xor_c(v[k1], s);
      const cpx<T> t = up ? csub(u, v[k1]) : cadd(v[k1], u);
      v[k1] = cmul(t, w);
    }
  }
}

__device__ __forceinline__ int out_index(int k1, int E, int lane) { return k1 + E * (int)(__brev((unsigned)lane) >> 27); }

// Shared scratch of the warp FFTs carries one padding slot per 32 elements
// (pencils) or per 32 rows (tiles): a warp's outputs, stored in bit-reversed
// order with index stride E, then fall into distinct banks (2 wavefronts per
// 8-byte warp store instead of 2E) while natural-order loads stay at 2.
__device__ __forceinline__ int zpad(int i) { return i + (i >> 5); }
__device__ __forceinline__ int tpad(int j, int LD, int c) { return j * LD + (j >> 5) + c; }
constexpr int padded_len(int n) { return n + n / 32; }

// ===========================================================================
// Group FFT (single precision).  A pencil of N = F Q points is transformed by
// Q lanes of a warp holding F values each, so one warp takes 32 / Q pencils at
// a time and the cross-lane part costs one exchange through shared memory
// instead of five shuffle stages.  With n = q + Q m and k = k1 + F k2
// (Cooley-Tukey):
//   1. F-point DFT over m in registers (radix 2, constant twiddles);
//   2. twiddle W_N^(q k1) from a lane-contiguous table;
//   3. exchange through the pencil's own shared-memory slots: value (k1, q')
//      goes to slot k1 Q + (q' ^ (k1 mod Q)); lane q then takes k1 = q + Q r
//      (r < F / Q), reads its Q values and does the Q-point DFT over q' in
//      registers.
// Lane q then holds X[q + Q r + F k2] in register r Q + k2.  The XOR swizzle
// keeps the exchange's stores (fixed k1, lanes q') and loads (fixed r and q',
// lanes q) on distinct banks within a group.
// ===========================================================================
template <int N> struct GroupShape;
template <> struct GroupShape<32> { static constexpr int F = 8, Q = 4; };
template <> struct GroupShape<64> { static constexpr int F = 8, Q = 8; };
template <> struct GroupShape<128> { static constexpr int F = 16, Q = 8; };
template <> struct GroupShape<256> { static constexpr int F = 16, Q = 16; };
// shared stride of a group's pencil slot: the G = 32 / Q groups of a warp
// then start 16 / G banks (of 8-byte entries) apart
template <int N> constexpr int group_ps() { return N + 16 / (32 / GroupShape<N>::Q); }
// Row passes (r2c / c2r of row pairs) by group FFTs: single precision at
// N = 256 (measured faster there; at N <= 128 the warp FFT's rows, whose warp
// loads and stores take whole 128-byte lines, measured faster).  Every kernel
// of one grid size takes the same choice, so all its paths give the same bits.
template <typename T, int N> constexpr bool group_rows() { return sizeof(T) == 4 && N == 256; }
// shared entries of a kernel's group-FFT twiddle table (single precision only)
template <typename T, int N> constexpr int twq_len() { return sizeof(T) == 4 ? N : 0; }

// v * W_16^t (forward: W = e^{-2 pi i / 16}; DIR > 0: the conjugate), t in
// [0, 8) a compile-time constant after unrolling: the quarter and eighth turns
// take no general product.
template <typename T, int DIR>
__device__ __forceinline__ cpx<T> rot16(cpx<T> v, int t) {
  const T c1 = T(0.92387953251128674), s1 = T(0.38268343236508977), h = T(0.70710678118654752);
  if (t == 0) return v;
  if (t == 4) return DIR < 0 ? cpx<T>{v.y, -v.x} : cpx<T>{-v.y, v.x};
  if (t == 2)
    return DIR < 0 ? cpx<T>{t_mul_rn(h, v.x + v.y), t_mul_rn(h, v.y - v.x)}
                   : cpx<T>{t_mul_rn(h, v.x - v.y), t_mul_rn(h, v.x + v.y)};
  if (t == 6)
    return DIR < 0 ? cpx<T>{t_mul_rn(h, v.y - v.x), -t_mul_rn(h, v.x + v.y)}
                   : cpx<T>{-t_mul_rn(h, v.x + v.y), t_mul_rn(h, v.x - v.y)};
  // odd t: cos and sin of 2 pi t / 16
  const T cs = (t == 1 || t == 7) ? c1 : s1, sn = (t == 1 || t == 7) ? s1 : c1;
  const T wr = t < 4 ? cs : -cs, wi = DIR < 0 ? -sn : sn;
  return cmul(v, cpx<T>{wr, wi});
}

__host__ __device__ constexpr int brev_c(int i, int lg) {
  int r = 0;
  for (int b = 0; b < lg; ++b) r |= ((i >> b) & 1) << (lg - 1 - b);
  return r;
}

// n-point DFT (n = 2, 4, 8, 16) of v[OFF .. OFF + n) in registers, natural
// order in and out: radix-2 decimation in time over the bit-reversed inputs.
template <typename T, int n, int DIR, int OFF, int LEN>
__device__ __forceinline__ void reg_fft(cpx<T> (&v)[LEN]) {
  constexpr int LG = n == 2 ? 1 : n == 4 ? 2 : n == 8 ? 3 : 4;
  cpx<T> a[n];
#pragma unroll
  for (int i = 0; i < n; ++i) a[brev_c(i, LG)] = v[OFF + i];
#pragma unroll
  for (int h = 1; h < n; h <<= 1)
#pragma unroll
    for (int g = 0; g < n; g += 2 * h)
#pragma unroll
      for (int k = 0; k < h; ++k) {
        const cpx<T> b = rot16<T, DIR>(a[g + k + h], k * (8 / h));   // W_{2h}^k = W_16^(8 k / h)
        const cpx<T> u = a[g + k];
        a[g + k] = cadd(u, b);
        a[g + k + h] = csub(u, b);
      }
#pragma unroll
  for (int i = 0; i < n; ++i) v[OFF + i] = a[i];
}

// The group FFT's twiddle table: twq[k1 Q + q] = W_N^(q k1), N entries.
template <typename T, int N> __device__ __forceinline__ void load_twq(cpx<T>* twq) {
  constexpr int Q = GroupShape<N>::Q;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int k1 = i / Q, q = i - k1 * Q;
    const int m = (q * k1 * (kNmax / N)) & (kNmax - 1);
    twq[i] = cpx<T>{(T)g_twiddle[m].x, (T)g_twiddle[m].y};
  }
}

// One pencil on the Q lanes of a group (q: lane within the group; mask: the
// lanes of the warp taking part).  On entry v[m] = x[q + Q m]; on return
// v[r Q + k2] = X[q + Q r + F k2].  slot(j) points at the pencil's element j
// in shared memory; its inputs must already be in registers (the slots are
// overwritten by the exchange), and every lane has finished with the slots
// when this returns.
template <typename T, int N, int DIR, typename Slot>
__device__ __forceinline__ void group_fft(cpx<T> (&v)[GroupShape<N>::F], int q, const cpx<T>* twq, unsigned mask,
                                          Slot slot) {
  constexpr int F = GroupShape<N>::F, Q = GroupShape<N>::Q, R = F / Q;
  reg_fft<T, F, DIR, 0>(v);
#pragma unroll
  for (int k1 = 1; k1 < F; ++k1) {
    cpx<T> w = twq[k1 * Q + q];
    if (DIR > 0) w.y = -w.y;
    v[k1] = cmul(v[k1], w);
  }
  __syncwarp(mask);
#pragma unroll
  for (int k1 = 0; k1 < F; ++k1) *slot(k1 * Q + (q ^ (k1 & (Q - 1)))) = v[k1];
  __syncwarp(mask);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int i = 0; i < Q; ++i) v[r * Q + i] = *slot((q + Q * r) * Q + (i ^ q));
  __syncwarp(mask);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r == 0) reg_fft<T, Q, DIR, 0>(v);
    if (r == 1) reg_fft<T, Q, DIR, Q>(v);
    if (r == 2) reg_fft<T, Q, DIR, 2 * Q>(v);
    if (r == 3) reg_fft<T, Q, DIR, 3 * Q>(v);
  }
}

// Task count for G pencils per warp task at pencil p = t + T g: the smallest
// T >= ceil(P / G) with T * S16 = 16 / G (mod 16), where S16 is the shared
// stride (complex entries, mod 16) between the storage of consecutive
// pencils, so the G groups of a warp start 16 / G banks apart.
template <int G>
__device__ __forceinline__ int spread_tasks(int P, int S16) {
  int t = (P + G - 1) / G;
  if (G > 2 && (S16 & 15))
    for (int i = 0; i < 16 && ((t * S16) & 15) != 16 / G; ++i) ++t;
  return t;
}

// Per-warp scratch of the row kernels (complex entries): single precision,
// one slot of XRegShape<N>::PS entries per group; double, one padded pencil.
template <typename T, int N> constexpr int row_scratch() {
  return group_rows<T, N>() ? (32 / GroupShape<N>::Q) * group_ps<N>() : N + N / 32;
}

// Row pairs r2c with group FFTs (single precision).  Pair pr: real rows 2 pr
// and 2 pr + 1 read as one complex pencil z = a + i b (load(pr, j, a, b)),
// transformed, and split into the half spectra A_k = (Z_k + conj Z_{N-k}) / 2
// and B_k = -i (Z_k - conj Z_{N-k}) / 2, k <= N / 2, handed to
// store(pr, k, A, B).  slot(pr, g) gives N shared entries for the pencil's
// exchange and split; every Z is read before store is called, so the
// destination rows themselves may serve.  S16: see spread_tasks.  (Staging
// each warp's row pairs through shared memory with whole-warp loads instead
// of the groups' 32-byte row segments measured slower.)
template <typename T, int N, typename Load, typename Slot, typename Store>
__device__ __forceinline__ void group_r2c_pairs(int npairs, int S16, const cpx<T>* twq, Load load, Slot slot,
                                                Store store) {
  constexpr int F = GroupShape<N>::F, Q = GroupShape<N>::Q, G = 32 / Q, R = F / Q, NH = N / 2 + 1;
  constexpr int KI = (NH + Q - 1) / Q;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  const int g = lane / Q, q = lane & (Q - 1);
  const int ntask = spread_tasks<G>(npairs, S16);
  for (int t = wib; t < ntask; t += nw) {
    const int pr = t + ntask * g;
    const bool valid = pr < npairs;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      cpx<T> v[F];
#pragma unroll
      for (int m = 0; m < F; ++m) load(pr, q + Q * m, v[m].x, v[m].y);
      cpx<T>* z = slot(pr, g);
      group_fft<T, N, -1>(v, q, twq, mask, [z](int j) { return z + j; });
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) z[q + Q * r + F * k2] = v[r * Q + k2];
      __syncwarp(mask);
      cpx<T> zk[KI], zm[KI];
#pragma unroll
      for (int i = 0; i < KI; ++i) {
        const int k = q + Q * i;
        if (k < NH) {
          zk[i] = z[k];
          zm[i] = cconj(z[(N - k) & (N - 1)]);
        }
      }
      __syncwarp(mask);
#pragma unroll
      for (int i = 0; i < KI; ++i) {
        const int k = q + Q * i;
        if (k < NH) {
          const cpx<T> d = csub(zk[i], zm[i]);
          store(pr, k, cpx<T>{(zk[i].x + zm[i].x) * T(0.5), (zk[i].y + zm[i].y) * T(0.5)},
                cpx<T>{d.y * T(0.5), -d.x * T(0.5)});
        }
      }
      __syncwarp(mask);
    }
  }
}

// Row pairs c2r with group FFTs (single precision).  Pair pr's Hermitian half
// rows A (row 2 pr) and B (row 2 pr + 1), k <= N / 2, from half(pr, k, A, B),
// become the pencil Z = A + i B (Z_k = A_k + i B_k, Z_{N-k} = conj A_k +
// i conj B_k), whose inverse transform gives row 2 pr as its real part and
// row 2 pr + 1 as its imaginary part: out(pr, j, re, im).  slot(pr, g): N
// shared entries (every half value is read before the slot is written, so
// the pair's own rows may serve).
template <typename T, int N, typename Half, typename Slot, typename Out>
__device__ __forceinline__ void group_c2r_pairs(int npairs, int S16, const cpx<T>* twq, Half half, Slot slot,
                                                Out out) {
  constexpr int F = GroupShape<N>::F, Q = GroupShape<N>::Q, G = 32 / Q, R = F / Q, NH = N / 2 + 1;
  constexpr int KI = (NH + Q - 1) / Q;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  const int g = lane / Q, q = lane & (Q - 1);
  const int ntask = spread_tasks<G>(npairs, S16);
  for (int t = wib; t < ntask; t += nw) {
    const int pr = t + ntask * g;
    const bool valid = pr < npairs;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      cpx<T> a[KI], b[KI];
#pragma unroll
      for (int i = 0; i < KI; ++i) {
        const int k = q + Q * i;
        if (k < NH) half(pr, k, a[i], b[i]);
      }
      cpx<T>* z = slot(pr, g);
      __syncwarp(mask);
#pragma unroll
      for (int i = 0; i < KI; ++i) {
        const int k = q + Q * i;
        if (k < NH) {
          cpx<T> A = a[i], B = b[i];
          if (k == 0 || k == N / 2) {
            A.y = T(0);
            B.y = T(0);
          }
          z[k] = cpx<T>{A.x - B.y, A.y + B.x};
          if (k > 0 && k < N / 2) z[N - k] = cpx<T>{A.x + B.y, -A.y + B.x};   // conj A + i conj B
        }
      }
      __syncwarp(mask);
      cpx<T> v[F];
#pragma unroll
      for (int m = 0; m < F; ++m) v[m] = z[q + Q * m];
      group_fft<T, N, +1>(v, q, twq, mask, [z](int j) { return z + j; });
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) out(pr, q + Q * r + F * k2, v[r * Q + k2].x, v[r * Q + k2].y);
      __syncwarp(mask);
    }
  }
}

// In-place FFTs of P pencils in shared memory (element j of pencil p at
// at(p, j); pencils with ok(p) false are left alone), spread over the block's
// warps.  Single precision: group FFTs, the G = 32 / Q pencils of warp task t
// at p = t, t + T, t + 2T, ...; with T = 16/G mod 32/G and pencils one bank
// apart (consecutive columns of a tile) the G groups start 16/G banks apart,
// so a warp's 8-byte accesses take two wavefronts (for G = 2 they do at any
// T).  Double precision: one pencil per warp (warp_fft).
template <typename T, int N, int DIR, typename At, typename Ok>
__device__ __forceinline__ void tile_ffts(int P, const cpx<T>* tw, const cpx<T>* twq, At at, Ok ok) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  if constexpr (sizeof(T) == 4) {
    constexpr int F = GroupShape<N>::F, Q = GroupShape<N>::Q, G = 32 / Q;
    const int g = lane / Q, q = lane & (Q - 1);
    constexpr int MOD = 32 / G, RES = 16 / G;
    int ntask = (P + G - 1) / G;
    // ntask = RES (mod MOD); two groups (N = 256) take two wavefronts anyway
    if (G > 2) ntask += ((RES - ntask) % MOD + MOD) % MOD;
    for (int t = wib; t < ntask; t += nw) {
      const int p = t + ntask * g;
      const bool valid = p < P && ok(p);
      const unsigned mask = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        cpx<T> v[F];
#pragma unroll
        for (int m = 0; m < F; ++m) v[m] = *at(p, q + Q * m);
        group_fft<T, N, DIR>(v, q, twq, mask, [&](int j) { return at(p, j); });
#pragma unroll
        for (int r = 0; r < F / Q; ++r)
#pragma unroll
          for (int k2 = 0; k2 < Q; ++k2) *at(p, q + Q * r + F * k2) = v[r * Q + k2];
      }
    }
  } else {
    constexpr int E = N / 32;
    for (int p = wib; p < P; p += nw) {
      if (!ok(p)) continue;
      cpx<T> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = *at(p, lane + 32 * m);
      warp_fft<T, E, DIR>(v, lane, tw);
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) *at(p, out_index(k1, E, lane)) = v[k1];
    }
  }
}

template <typename T, int E> __device__ __forceinline__ void load_tw_full(cpx<T>* tw) {
  constexpr int SC = kNmax / (32 * E);
  for (int i = threadIdx.x; i < kNmax + 32 * E; i += blockDim.x) {
    int m;
    if (i < kNmax) {
      m = i;
    } else if (i < kNmax + 32) {   // stage s = 2^floor(log2 j), j - s = lane mod s (entry kNmax: unused, 1)
      const int j = i - kNmax;
      const int st = 1 << (31 - __clz(j | 1));
      m = j == 0 ? 0 : (j - st) * (kNmax / (2 * st));
    } else {
      const int j = i - kNmax, k1 = j >> 5, lane = j & 31;
      m = (lane * k1 * SC) & (kNmax - 1);
    }
    tw[i] = cpx<T>{(T)g_twiddle[m].x, (T)g_twiddle[m].y};
  }
}

// Shared twiddles of a kernel whose column passes use tile_ffts: the warp
// FFT's tables (kTwLen entries), then, in single precision, the group FFT's.
template <typename T, int E> constexpr int tw_len() { return kTwLen + twq_len<T, 32 * E>(); }
template <typename T, int E> __device__ __forceinline__ void load_tw_group(cpx<T>* tw) {
  load_tw_full<T, E>(tw);
  if constexpr (sizeof(T) == 4) load_twq<T, 32 * E>(tw + kTwLen);
}


// Kernel bodies take their arrays and block coordinates explicitly so the same
// code serves one run (the __global__ wrappers below) and a batch of runs
// (the *_batch kernels, one run per block row).

// Rows r2c: each warp takes row pairs (two real rows as one complex pencil).
template <typename T, int E, typename Tin>
__device__ __forceinline__ void rows_r2c_body(Tin* __restrict__ in, double in_scale, int zero_input,
                                              cpx<T>* __restrict__ out, int rows, double* mass_acc, int bx, int gx,
                                              const cpx<T>* tw, cpx<T>* zball) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cpx<T>* zb = zball + wib * row_scratch<T, N>();
  double msum = 0.0;
  if constexpr (group_rows<T, N>()) {
    // group FFTs over this block's contiguous range of row pairs
    constexpr int PS = group_ps<N>();
    const int np = rows / 2, per = (np + gx - 1) / gx, p0 = bx * per, cnt = max(0, min(per, np - p0));
    group_r2c_pairs<T, N>(
        cnt, 0, tw + kTwLen,
        [&](int pr, int j, T& a, T& b) {
          const size_t ra = (size_t)(2 * (p0 + pr)) * N + j, rb = ra + N;
          if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value) {
            a = (T)((double)(long long)in[ra] * in_scale);
            b = (T)((double)(long long)in[rb] * in_scale);
          } else {
            a = (T)in[ra];
            b = (T)in[rb];
          }
          if (zero_input) {
            in[ra] = Tin(0);
            in[rb] = Tin(0);
          }
          if (mass_acc) msum += (double)a + (double)b;
        },
        [&](int, int g) { return zb + g * PS; },
        [&](int pr, int k, cpx<T> A, cpx<T> B) {
          cpx<T>* oa = out + (size_t)(2 * (p0 + pr)) * NH;
          oa[k] = A;
          oa[NH + k] = B;
        });
  } else {
  const int nwarps = gx * 8;
  for (int pr = bx * 8 + wib; pr < rows / 2; pr += nwarps) {
    const size_t ra = (size_t)(2 * pr) * N, rb = ra + N;
    cpx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      T a, b;
      if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value) {
        a = (T)((double)(long long)in[ra + lane + 32 * m] * in_scale);
        b = (T)((double)(long long)in[rb + lane + 32 * m] * in_scale);
      } else {
        a = (T)in[ra + lane + 32 * m];
        b = (T)in[rb + lane + 32 * m];
      }
      v[m] = cpx<T>{a, b};
    }
    if (zero_input) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        in[ra + lane + 32 * m] = Tin(0);
        in[rb + lane + 32 * m] = Tin(0);
      }
    }
    if (mass_acc) {
#pragma unroll
      for (int m = 0; m < E; ++m) msum += (double)v[m].x + (double)v[m].y;
    }
    warp_fft<T, E, -1>(v, lane, tw);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) zb[zpad(out_index(k1, E, lane))] = v[k1];
    __syncwarp();
    cpx<T>* oa = out + (size_t)(2 * pr) * NH;
    for (int k = lane; k < NH; k += 32) {
      const cpx<T> zk = zb[zpad(k)];
      const cpx<T> zm = cconj(zb[zpad((N - k) & (N - 1))]);
      const cpx<T> d = csub(zk, zm);
      oa[k] = cpx<T>{(zk.x + zm.x) * T(0.5), (zk.y + zm.y) * T(0.5)};
      oa[NH + k] = cpx<T>{d.y * T(0.5), -d.x * T(0.5)};
    }
    __syncwarp();
  }
  }
  if (mass_acc) {
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, o);
    if (lane == 0) atomicAdd(mass_acc, msum);
  }
}

template <typename T, int E, typename Tin>
__global__ void __launch_bounds__(256)
kw_rows_r2c(Tin* __restrict__ in, double in_scale, int zero_input, cpx<T>* __restrict__ out, int rows,
            double* mass_acc) {
  __shared__ cpx<T> tw[tw_len<T, E>()];
  __shared__ cpx<T> zb[8 * row_scratch<T, 32 * E>()];
  load_tw_group<T, E>(tw);
  __syncthreads();
  rows_r2c_body<T, E, Tin>(in, in_scale, zero_input, out, rows, mass_acc, blockIdx.x, gridDim.x, tw, zb);
}

// c2c along the middle axis of [A][H][B]: a block stages an H x BC tile
// (coalesced row segments), warps transform its columns from shared memory.
template <typename T, int E, int DIR, int BC>
__device__ __forceinline__ void cols_body(cpx<T>* __restrict__ base, int B, T scale, int b0, const cpx<T>* tw,
                                          cpx<T>* buf) {
  constexpr int N = 32 * E, LD = BC + 1;
  const int nb = min(BC, B - b0);
  for (int t = threadIdx.x; t < N * BC; t += blockDim.x) {
    const int j = t / BC, c = t - j * BC;
    buf[tpad(j, LD, c)] = c < nb ? base[(size_t)j * B + b0 + c] : cpx<T>{T(0), T(0)};
  }
  __syncthreads();
  tile_ffts<T, N, DIR>(nb, tw, tw + kTwLen, [&](int p, int j) { return buf + tpad(j, LD, p); },
                       [](int) { return true; });
  __syncthreads();
  for (int t = threadIdx.x; t < N * BC; t += blockDim.x) {
    const int j = t / BC, c = t - j * BC;
    if (c < nb) {
      const cpx<T> v = buf[tpad(j, LD, c)];
      base[(size_t)j * B + b0 + c] = cpx<T>{v.x * scale, v.y * scale};
    }
  }
}

template <typename T, int E, int DIR, int BC>
__global__ void __launch_bounds__(256)
kw_cols(cpx<T>* __restrict__ data, int B, size_t comp_stride, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  load_tw_group<T, E>(tw);
  cpx<T>* base = data + blockIdx.z * comp_stride + (size_t)blockIdx.y * (32 * E) * B;
  cols_body<T, E, DIR, BC>(base, B, scale, blockIdx.x * BC, tw, tw + tw_len<T, E>());
}

// x-axis pass fused with the spectral work (as k_spectral_x), warp FFTs.
// Shared tile: [N][3 BC + 1]; slot 0 = beta, then the first output (each
// element's beta is read before its outputs are written), slots 1, 2 the other
// two outputs: 3 slots per pencil, so a 128^3 x pass fits one wave of blocks.
template <typename T, int E, int MODE, int BC>
__device__ __forceinline__ void spectral_body(const cpx<T>* __restrict__ T1, cpx<T>* __restrict__ alpha,
                                              cpx<T>* __restrict__ T2, const SpecParams& sp, double* alpha0_shadow,
                                              int b0, const cpx<T>* tw, const cpx<T>* twq, cpx<T>* buf) {
  constexpr int N = 32 * E, NHH = N / 2 + 1, LD = 3 * BC + 1;
  const int B = N * NHH;
  const size_t S = (size_t)N * B;
  const int nb = min(BC, B - b0);
  constexpr bool needs_beta = (MODE == kModeStep || MODE == kModeDensity);
  if (needs_beta) {
    for (int t = threadIdx.x; t < N * BC; t += blockDim.x) {
      const int j = t / BC, c = t - j * BC;
      buf[tpad(j, LD, c)] = c < nb ? T1[(size_t)j * B + b0 + c] : cpx<T>{T(0), T(0)};
    }
    __syncthreads();
    tile_ffts<T, N, -1>(nb, tw, twq, [&](int p, int j) { return buf + tpad(j, LD, p); }, [](int) { return true; });
  }
  __syncthreads();
  const T two_pi_L = (T)(2.0 * M_PI / sp.L);
  const T inv_L3 = (T)sp.inv_L3;
  const T tau_eps = (T)(sp.tau / sp.eps), eps_tau = (T)(sp.eps / sp.tau), k2 = (T)sp.k2, tau = (T)sp.tau;
  const T filt = sp.H0 > 0 ? (T)(-2.0 * M_PI * M_PI / (sp.H0 * sp.H0)) : T(0);
  for (int t = threadIdx.x; t < N * BC; t += blockDim.x) {
    const int j = t / BC, c = t - j * BC;
    const int m = b0 + c;
    cpx<T> o1{T(0), T(0)}, o2{T(0), T(0)}, o3{T(0), T(0)};
    if (c < nb) {
      const int ky = m / NHH, kz = m - ky * NHH;
      const int qx = j < N / 2 ? j : j - N;
      const int qy = ky < N / 2 ? ky : ky - N;
      const int qz = kz < N / 2 ? kz : kz - N;
      const T q2 = (T)(qx * qx + qy * qy + qz * qz);
      const T Phi = sp.H0 > 0 ? t_exp(filt * q2) : T(1);
      const size_t gi = (size_t)j * B + m;
      if (MODE == kModeStep || MODE == kModeGradOnly) {
        const cpx<T> a = alpha[gi];
        if (MODE == kModeStep) {
          cpx<T> beta = buf[tpad(j, LD, c)];
          beta.x *= inv_L3;
          beta.y *= inv_L3;
          const T lam = two_pi_L * two_pi_L * q2 + k2;
          cpx<T> an;
          if (sp.propagator == 0) {
            const T kappa = T(1) / (T(1) + tau_eps * lam);
            const T src = T(1) / (lam + eps_tau);
            an = cpx<T>{kappa * a.x + src * beta.x, kappa * a.y + src * beta.y};
          } else {
            const T kappa = t_exp(-tau_eps * lam);
            an = cpx<T>{kappa * (a.x + tau * beta.x), kappa * (a.y + tau * beta.y)};
          }
          alpha[gi] = an;
          if (m == 0 && j == 0 && alpha0_shadow) {
            const double lam0 = sp.k2;
            double s = *alpha0_shadow;
            if (sp.propagator == 0) s = s / (1.0 + sp.tau / sp.eps * lam0) + sp.beta0 / (lam0 + sp.eps / sp.tau);
            else s = exp(-sp.tau / sp.eps * lam0) * (s + sp.tau * sp.beta0);
            *alpha0_shadow = s;
          }
        }
        const T yx = two_pi_L * (T)qx * Phi, yy = two_pi_L * (T)qy * Phi, yz = two_pi_L * (T)qz * Phi;
        if (qx != -N / 2) o1 = cpx<T>{-yx * a.y, yx * a.x};
        if (qy != -N / 2) o2 = cpx<T>{-yy * a.y, yy * a.x};
        if (qz != -N / 2) o3 = cpx<T>{-yz * a.y, yz * a.x};
      } else if (MODE == kModeDensity) {
        const cpx<T> beta = buf[tpad(j, LD, c)];
        o1 = cpx<T>{beta.x * inv_L3 * Phi, beta.y * inv_L3 * Phi};
      } else {
        o1 = alpha[gi];
      }
    }
    buf[tpad(j, LD, c)] = o1;
    buf[tpad(j, LD, BC + c)] = o2;
    buf[tpad(j, LD, 2 * BC + c)] = o3;
  }
  __syncthreads();
  constexpr int nout = (MODE == kModeStep || MODE == kModeGradOnly) ? 3 : 1;
  tile_ffts<T, N, +1>(nout * BC, tw, twq, [&](int p, int j) { return buf + tpad(j, LD, p); },
                      [&](int p) { return p % BC < nb; });
  __syncthreads();
  for (int t = threadIdx.x; t < N * BC; t += blockDim.x) {
    const int j = t / BC, c = t - j * BC;
    if (c < nb) {
#pragma unroll
      for (int d = 0; d < nout; ++d) T2[d * S + (size_t)j * B + b0 + c] = buf[tpad(j, LD, d * BC + c)];
    }
  }
}

// ---------------------------------------------------------------------------
// Single-precision x pass in registers.  A warp takes G = 32 / Q consecutive
// pencils (m0 .. m0 + G - 1, x along each; element j of pencil m at j B + m);
// lane q of group g keeps its pencil's elements j = q + Q s (s < F) in
// registers from the global load, through the forward group FFT, the
// spectral update and the inverse group FFTs to the global store, so no
// block-wide barrier is needed.  The old alpha comes in by cp.async into a
// per-warp slot while beta is transformed.  The three gradient spectra take
// two inverse transforms: q_y and q_z are constant along an x pencil, so
// G_y and G_z are i (2 pi q_d / L) times the x-inverse of Phi alpha; only
// G_x needs its own.
// ---------------------------------------------------------------------------
template <int N> struct XRegShape {
  static constexpr int F = GroupShape<N>::F, Q = GroupShape<N>::Q, G = 32 / Q;
  static constexpr int PS = group_ps<N>();  // pencil stride in a warp slot
  static constexpr int WARP = 2 * G * PS;   // complex entries per warp: exchange slots + alpha slots
  static constexpr int TASKS = N * (N / 2 + 1) / G;
  static_assert(N * (N / 2 + 1) % G == 0, "x pencils come in whole groups");
};
template <int N> constexpr size_t xreg_smem_bytes(int nw) {
  return ((size_t)N + (size_t)nw * XRegShape<N>::WARP) * sizeof(cpx<float>);
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int N, int MODE>
__device__ __forceinline__ void spectral_reg_task(const cpx<float>* __restrict__ T1, cpx<float>* __restrict__ alpha,
                                                  cpx<float>* __restrict__ T2, const SpecParams& sp,
                                                  double* alpha0_shadow, int m0, const cpx<float>* twq,
                                                  cpx<float>* wslot) {
  using S = XRegShape<N>;
  constexpr int F = S::F, Q = S::Q, R = F / Q, NHH = N / 2 + 1, B = N * NHH;
  constexpr size_t SZ = (size_t)N * B;
  constexpr bool reads_alpha = MODE != kModeDensity;
  constexpr bool needs_beta = MODE == kModeStep || MODE == kModeDensity;
  constexpr bool grad = MODE == kModeStep || MODE == kModeGradOnly;
  const int lane = threadIdx.x & 31, g = lane / Q, q = lane & (Q - 1);
  const int m = m0 + g;
  cpx<float>* X = wslot + g * S::PS;              // this pencil's exchange slots
  cpx<float>* A = wslot + (S::G + g) * S::PS;     // its old alpha, then Phi alpha
  auto xs = [X](int j) { return X + j; };
  if (reads_alpha) {
#pragma unroll
    for (int s = 0; s < F; ++s) cp_async8(A + q + Q * s, alpha + (size_t)(q + Q * s) * B + m);
  }
  const int ky = m / NHH, kz = m - ky * NHH;
  const int qy = ky < N / 2 ? ky : ky - N, qz = kz < N / 2 ? kz : kz - N;
  const float two_pi_L = (float)(2.0 * M_PI / sp.L);
  const float inv_L3 = (float)sp.inv_L3;
  const float tau_eps = (float)(sp.tau / sp.eps), eps_tau = (float)(sp.eps / sp.tau), k2 = (float)sp.k2,
              tau = (float)sp.tau;
  const float filt = sp.H0 > 0 ? (float)(-2.0 * M_PI * M_PI / (sp.H0 * sp.H0)) : 0.f;
  cpx<float> v[F];
  if (needs_beta) {
#pragma unroll
    for (int s = 0; s < F; ++s) v[s] = T1[(size_t)(q + Q * s) * B + m];
    group_fft<float, N, -1>(v, q, twq, 0xffffffffu, xs);   // v[r Q + k2] = beta^[q + Q (r + R k2)]
  }
  if (reads_alpha) cp_async_wait_all();
  cpx<float> w[F];   // the first inverse transform's input, element q + Q s at w[s]
#pragma unroll
  for (int s = 0; s < F; ++s) {
    const int j = q + Q * s;
    const int qx = j < N / 2 ? j : j - N;
    const float q2 = (float)(qx * qx + qy * qy + qz * qz);
    const float Phi = sp.H0 > 0 ? expf(filt * q2) : 1.f;
    cpx<float> o1{0.f, 0.f};
    if (grad) {
      const cpx<float> a = A[q + Q * s];
      if (MODE == kModeStep) {
        cpx<float> beta = v[(s % R) * Q + s / R];
        beta.x *= inv_L3;
        beta.y *= inv_L3;
        const float lam = two_pi_L * two_pi_L * q2 + k2;
        cpx<float> an;
        if (sp.propagator == 0) {
          const float kappa = 1.f / (1.f + tau_eps * lam);
          const float src = 1.f / (lam + eps_tau);
          an = cpx<float>{kappa * a.x + src * beta.x, kappa * a.y + src * beta.y};
        } else {
          const float kappa = expf(-tau_eps * lam);
          an = cpx<float>{kappa * (a.x + tau * beta.x), kappa * (a.y + tau * beta.y)};
        }
        alpha[(size_t)j * B + m] = an;
        if (m == 0 && j == 0 && alpha0_shadow) {
          const double lam0 = sp.k2;
          double sh = *alpha0_shadow;
          if (sp.propagator == 0) sh = sh / (1.0 + sp.tau / sp.eps * lam0) + sp.beta0 / (lam0 + sp.eps / sp.tau);
          else sh = exp(-sp.tau / sp.eps * lam0) * (sh + sp.tau * sp.beta0);
          *alpha0_shadow = sh;
        }
      }
      const float yx = two_pi_L * (float)qx * Phi;
      if (qx != -N / 2) o1 = cpx<float>{-yx * a.y, yx * a.x};
      A[q + Q * s] = cpx<float>{Phi * a.x, Phi * a.y};
    } else if (MODE == kModeDensity) {
      const cpx<float> beta = v[(s % R) * Q + s / R];
      o1 = cpx<float>{beta.x * inv_L3 * Phi, beta.y * inv_L3 * Phi};
    } else {
      o1 = A[q + Q * s];
    }
    w[s] = o1;
  }
  group_fft<float, N, +1>(w, q, twq, 0xffffffffu, xs);
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int k = 0; k < Q; ++k) T2[(size_t)(q + Q * (r + R * k)) * B + m] = w[r * Q + k];
  if (grad) {
#pragma unroll
    for (int s = 0; s < F; ++s) w[s] = A[q + Q * s];
    group_fft<float, N, +1>(w, q, twq, 0xffffffffu, xs);
    const float cy = qy != -N / 2 ? two_pi_L * (float)qy : 0.f, cz = qz != -N / 2 ? two_pi_L * (float)qz : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        const size_t gi = (size_t)(q + Q * (r + R * k)) * B + m;
        const cpx<float> u = w[r * Q + k];
        T2[SZ + gi] = cpx<float>{-cy * u.y, cy * u.x};
        T2[2 * SZ + gi] = cpx<float>{-cz * u.y, cz * u.x};
      }
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(256)
kwr_spectral_x(const cpx<float>* __restrict__ T1, cpx<float>* __restrict__ alpha, cpx<float>* __restrict__ T2,
               SpecParams sp, double* alpha0_shadow) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* twq = reinterpret_cast<cpx<float>*>(smem_raw);
  load_twq<float, N>(twq);
  __syncthreads();
  const int wib = threadIdx.x >> 5;
  const int t = blockIdx.x * (int)(blockDim.x >> 5) + wib;
  if (t < XRegShape<N>::TASKS)
    spectral_reg_task<N, MODE>(T1, alpha, T2, sp, alpha0_shadow, t * XRegShape<N>::G, twq,
                               twq + N + wib * XRegShape<N>::WARP);
}

template <int N>
__global__ void __launch_bounds__(512) kwrb_spectral_x(const FftRun<float>* __restrict__ runs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* twq = reinterpret_cast<cpx<float>*>(smem_raw);
  load_twq<float, N>(twq);
  __syncthreads();
  const FftRun<float>& r = runs[blockIdx.y];
  const int wib = threadIdx.x >> 5;
  const int t = blockIdx.x * (int)(blockDim.x >> 5) + wib;
  if (t < XRegShape<N>::TASKS)
    spectral_reg_task<N, kModeStep>(r.T1, r.alpha, r.T2, r.sp, r.shadow, t * XRegShape<N>::G, twq,
                                    twq + N + wib * XRegShape<N>::WARP);
}

template <typename T, int E, int MODE, int BC>
__global__ void __launch_bounds__(256)
kw_spectral_x(const cpx<T>* __restrict__ T1, cpx<T>* __restrict__ alpha, cpx<T>* __restrict__ T2, SpecParams sp,
              double* alpha0_shadow) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  load_tw_full<T, E>(tw);
  cpx<T>* twq = tw + kTwLen;
  if constexpr (sizeof(T) == 4) load_twq<T, 32 * E>(twq);
  spectral_body<T, E, MODE, BC>(T1, alpha, T2, sp, alpha0_shadow, blockIdx.x * BC, tw, twq,
                                twq + twq_len<T, 32 * E>());
}

// Rows c2r: each warp takes a row pair of every component, rebuilds the
// full pencil Z = A + i B from the Hermitian halves, inverse-transforms it,
// and writes (gx, gy, gz, 0) nodes (NCOMP == 3) or a plain grid (NCOMP == 1).
template <typename T, int E, int NCOMP>
__device__ __forceinline__ void rows_c2r_body(const cpx<T>* __restrict__ in, size_t comp_stride, T* __restrict__ out,
                                              int rows, double* max_acc, int bx, int gx, const cpx<T>* tw,
                                              cpx<T>* zb_all, T* ob_all) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  constexpr int NOUT = NCOMP == 3 ? 4 : 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cpx<T>* zb = zb_all + wib * row_scratch<T, N>();
  double mx = -INFINITY;
  if constexpr (group_rows<T, N>()) {
    // group FFTs over this block's contiguous range of row pairs, taken in
    // chunks of one pass of the block's warps, each chunk's components one
    // after another: a node's three components are written within a few
    // microseconds, so L2 merges the partial sectors before they go to DRAM
    // (whole components one after another left 1.9x the algorithmic traffic)
    constexpr int PS = group_ps<N>();
    const int np = rows / 2, per = (np + gx - 1) / gx, p0 = bx * per, cnt = max(0, min(per, np - p0));
    const int chunk = (int)(blockDim.x >> 5) * (32 / GroupShape<N>::Q);
    for (int c0 = 0; c0 < cnt; c0 += chunk) {
      const int cc = min(chunk, cnt - c0), q0 = p0 + c0;
      for (int d = 0; d < NCOMP; ++d) {
        const cpx<T>* src = in + d * comp_stride;
        group_c2r_pairs<T, N>(
            cc, 0, tw + kTwLen,
            [&](int pr, int k, cpx<T>& A, cpx<T>& B) {
              const cpx<T>* ra = src + (size_t)(2 * (q0 + pr)) * NH;
              A = ra[k];
              B = ra[NH + k];
            },
            [&](int, int g) { return zb + g * PS; },
            [&](int pr, int j, T re, T im) {
              T* oa = out + (size_t)(2 * (q0 + pr)) * N * NOUT;
              if (NOUT == 4) {
                oa[(size_t)j * 4 + d] = re;
                oa[(size_t)(N + j) * 4 + d] = im;
              } else {
                oa[j] = re;
                oa[N + j] = im;
                mx = fmax(mx, fmax((double)re, (double)im));
              }
            });
      }
    }
  } else {
  T* ob = ob_all + wib * 2 * N * NOUT;
  const int nwarps = gx * 8;
  for (int pr = bx * 8 + wib; pr < rows / 2; pr += nwarps) {
    for (int d = 0; d < NCOMP; ++d) {
      const cpx<T>* ra = in + d * comp_stride + (size_t)(2 * pr) * NH;
      const cpx<T>* rb = ra + NH;
      for (int k = lane; k < NH; k += 32) {
        cpx<T> A = ra[k], Bv = rb[k];
        if (k == 0 || k == N / 2) {
          A.y = T(0);
          Bv.y = T(0);
        }
        zb[zpad(k)] = cpx<T>{A.x - Bv.y, A.y + Bv.x};
        if (k > 0 && k < N / 2) zb[zpad(N - k)] = cpx<T>{A.x + Bv.y, -A.y + Bv.x};   // conj A + i conj B
      }
      __syncwarp();
      cpx<T> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = zb[zpad(lane + 32 * m)];
      __syncwarp();
      warp_fft<T, E, +1>(v, lane, tw);
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) {
        const int j = out_index(k1, E, lane);
        ob[(0 * N + j) * NOUT + d] = v[k1].x;
        ob[(1 * N + j) * NOUT + d] = v[k1].y;
      }
    }
    __syncwarp();
    T* oa = out + (size_t)(2 * pr) * N * NOUT;
    if (NOUT == 4) {
      for (int t = lane; t < 2 * N; t += 32) {
        const T* sv = ob + t * 4;
        if constexpr (sizeof(T) == 4) {
          reinterpret_cast<float4*>(oa)[t] = make_float4(sv[0], sv[1], sv[2], 0.f);
        } else {
          reinterpret_cast<double2*>(oa)[2 * t] = make_double2(sv[0], sv[1]);
          reinterpret_cast<double2*>(oa)[2 * t + 1] = make_double2(sv[2], 0.0);
        }
      }
    } else {
      for (int t = lane; t < 2 * N; t += 32) {
        const T v = ob[t];
        oa[t] = v;
        mx = fmax(mx, (double)v);
      }
    }
    __syncwarp();
  }
  }
  if (NOUT == 1 && max_acc) {
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      long long b = __double_as_longlong(mx);
      if (b < 0) b ^= 0x7fffffffffffffffLL;
      atomicMax(reinterpret_cast<long long*>(max_acc), b);
    }
  }
}

template <typename T, int E, int NCOMP>
__global__ void __launch_bounds__(256)
kw_rows_c2r(const cpx<T>* __restrict__ in, size_t comp_stride, T* __restrict__ out, int rows, double* max_acc) {
  constexpr int N = 32 * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb_all = tw + tw_len<T, E>();
  T* ob_all = reinterpret_cast<T*>(zb_all + 8 * row_scratch<T, N>());
  load_tw_group<T, E>(tw);
  __syncthreads();
  rows_c2r_body<T, E, NCOMP>(in, comp_stride, out, rows, max_acc, blockIdx.x, gridDim.x, tw, zb_all, ob_all);
}

// ---------------------------------------------------------------------------
// Batched step kernels: runs of one grid size H, one run per block row (y or
// z), arrays and parameters from a device table.
// ---------------------------------------------------------------------------
template <typename T, int E>
__global__ void __launch_bounds__(256) kwb_rows_r2c(const FftRun<T>* __restrict__ runs) {
  __shared__ cpx<T> tw[tw_len<T, E>()];
  __shared__ cpx<T> zb[8 * row_scratch<T, 32 * E>()];
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.y];
  constexpr int N = 32 * E;
  if (r.phi_fixed)
    rows_r2c_body<T, E, unsigned long long>((unsigned long long*)r.phi, r.in_scale, 1, r.T1, N * N, nullptr,
                                            blockIdx.x, gridDim.x, tw, zb);
  else
    rows_r2c_body<T, E, T>((T*)r.phi, 1.0, 1, r.T1, N * N, nullptr, blockIdx.x, gridDim.x, tw, zb);
}

// which = 0: forward y pass of T1; 1: inverse y pass of the three T2 components
template <typename T, int E, int DIR, int BC>
__global__ void __launch_bounds__(256) kwb_cols(const FftRun<T>* __restrict__ runs, int ncomp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  load_tw_group<T, E>(tw);
  constexpr int N = 32 * E, NHH = N / 2 + 1;
  const int run = blockIdx.z / ncomp, comp = blockIdx.z - run * ncomp;
  const FftRun<T>& r = runs[run];
  const size_t S = (size_t)N * N * NHH;
  cpx<T>* data = DIR < 0 ? r.T1 : r.T2 + comp * S;
  cols_body<T, E, DIR, BC>(data + (size_t)blockIdx.y * N * NHH, NHH, T(1), blockIdx.x * BC, tw, tw + tw_len<T, E>());
}

template <typename T, int E, int BC>
__global__ void __launch_bounds__(512) kwb_spectral_x(const FftRun<T>* __restrict__ runs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  load_tw_full<T, E>(tw);
  cpx<T>* twq = tw + kTwLen;
  if constexpr (sizeof(T) == 4) load_twq<T, 32 * E>(twq);
  const FftRun<T>& r = runs[blockIdx.y];
  spectral_body<T, E, kModeStep, BC>(r.T1, r.alpha, r.T2, r.sp, r.shadow, blockIdx.x * BC, tw, twq,
                                     twq + twq_len<T, 32 * E>());
}

template <typename T, int E>
__global__ void __launch_bounds__(256) kwb_rows_c2r(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb_all = tw + tw_len<T, E>();
  T* ob_all = reinterpret_cast<T*>(zb_all + 8 * row_scratch<T, N>());
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.y];
  const size_t S = (size_t)N * N * (N / 2 + 1);
  rows_c2r_body<T, E, 3>(r.T2, S, r.grad, N * N, nullptr, blockIdx.x, gridDim.x, tw, zb_all, ob_all);
}

// Shared bytes of the row c2r kernels: twiddles, per-warp scratch and, in
// double precision, per-warp staging of the output rows.
template <typename T, int E, int NOUT> constexpr size_t row_c2r_smem() {
  return ((size_t)tw_len<T, E>() + (size_t)8 * row_scratch<T, 32 * E>()) * sizeof(cpx<T>) +
         (group_rows<T, 32 * E>() ? 0 : (size_t)8 * 2 * 32 * E * NOUT * sizeof(T));
}

// ---------------------------------------------------------------------------
// Plane kernels (H <= 128): one block holds a whole x-plane of the half
// spectrum, H x (H/2+1) complex values, in shared memory and does both inner
// axes there, so the y pass costs no extra trip through L2.
//   forward: r2c of the plane's rows (two real rows per complex warp FFT, the
//            deposit grid cleared as it is read), then the y-axis FFT of every
//            column, then one coalesced write of the plane;
//   inverse: one component's plane, y-axis inverse of every column, then c2r
//            of row pairs, written into that component's slot of the
//            interleaved (gx, gy, gz, -) nodes.
// ---------------------------------------------------------------------------
constexpr int kDefaultPlaneWarps = 8;      // warps per block of the plane kernels
constexpr int kDefaultSpectralWarps = 8;   // warps per block of the fused x pass

template <typename T, int E> constexpr size_t plane_smem_bytes(int nw) {
  // plane: H rows of H/2+1 plus one slot per 32 rows; one padded pencil per warp
  return ((size_t)32 * E * (16 * E + 1) + E + (group_rows<T, 32 * E>() ? 0 : (size_t)nw * padded_len(32 * E)) +
          tw_len<T, E>()) *
         sizeof(cpx<T>);
}

template <typename T, int E, typename Tin>
__device__ __forceinline__ void plane_fwd_body(Tin* __restrict__ in, double in_scale, cpx<T>* __restrict__ out,
                                               const cpx<T>* tw, cpx<T>* P, cpx<T>* zball) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cpx<T>* zb = zball + wib * padded_len(N);
  const int nw = (int)(blockDim.x >> 5);
  // 1. rows: two real rows as one complex pencil, split into their half
  //    spectra.  In single precision the raw values of a warp's next row
  //    pair are loaded one iteration ahead, so their latency overlaps this
  //    pair's transform (in double precision the extra registers spill).
  if constexpr (group_rows<T, N>()) {
    // group FFTs, each row pair transformed and split in its own rows of P
    group_r2c_pairs<T, N>(
        N / 2, 2 * NH, tw + kTwLen,
        [&](int pr, int j, T& a, T& b) {
          const size_t ra = (size_t)(2 * pr) * N + j, rb = ra + N;
          const Tin va = in[ra], vb = in[rb];
          in[ra] = Tin(0);
          in[rb] = Tin(0);
          if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value) {
            a = (T)((double)(long long)va * in_scale);
            b = (T)((double)(long long)vb * in_scale);
          } else {
            a = (T)va;
            b = (T)vb;
          }
        },
        [&](int pr, int) { return P + tpad(2 * pr, NH, 0); },
        [&](int pr, int k, cpx<T> A, cpx<T> B) {
          cpx<T>* pa = P + tpad(2 * pr, NH, 0);
          pa[k] = A;
          pa[NH + k] = B;
        });
  } else {
  constexpr bool PF = sizeof(T) == 4;
  Tin na[E], nb[E];
  if (PF && wib < N / 2) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      na[m] = in[(size_t)(2 * wib) * N + lane + 32 * m];
      nb[m] = in[(size_t)(2 * wib + 1) * N + lane + 32 * m];
    }
  }
  for (int pr = wib; pr < N / 2; pr += nw) {
    const size_t ra = (size_t)(2 * pr) * N, rb = ra + N;
    Tin ca[E], cb[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      ca[m] = PF ? na[m] : in[ra + lane + 32 * m];
      cb[m] = PF ? nb[m] : in[rb + lane + 32 * m];
    }
    if (PF && pr + nw < N / 2) {
      const size_t qa = (size_t)(2 * (pr + nw)) * N, qb = qa + N;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        na[m] = in[qa + lane + 32 * m];
        nb[m] = in[qb + lane + 32 * m];
      }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
      in[ra + lane + 32 * m] = Tin(0);
      in[rb + lane + 32 * m] = Tin(0);
    }
    cpx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value)
        v[m] = cpx<T>{(T)((double)(long long)ca[m] * in_scale), (T)((double)(long long)cb[m] * in_scale)};
      else
        v[m] = cpx<T>{(T)ca[m], (T)cb[m]};
    }
    warp_fft<T, E, -1>(v, lane, tw);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) zb[zpad(out_index(k1, E, lane))] = v[k1];
    __syncwarp();
    cpx<T>* pa = P + tpad(2 * pr, NH, 0);   // rows 2 pr and 2 pr + 1 are adjacent
    for (int k = lane; k < NH; k += 32) {
      const cpx<T> zk = zb[zpad(k)];
      const cpx<T> zm = cconj(zb[zpad((N - k) & (N - 1))]);
      const cpx<T> d = csub(zk, zm);
      pa[k] = cpx<T>{(zk.x + zm.x) * T(0.5), (zk.y + zm.y) * T(0.5)};
      pa[NH + k] = cpx<T>{d.y * T(0.5), -d.x * T(0.5)};
    }
    __syncwarp();
  }
  }
  __syncthreads();
  // 2. y axis: the plane's columns in place
  tile_ffts<T, N, -1>(NH, tw, tw + kTwLen, [&](int p, int j) { return P + tpad(j, NH, p); },
                      [](int) { return true; });
  __syncthreads();
  for (int t = threadIdx.x; t < N * NH; t += blockDim.x) out[t] = P[t + ((t / NH) >> 5)];
}

template <typename T, int E>
__device__ __forceinline__ void plane_inv_body(const cpx<T>* __restrict__ in, T* __restrict__ out, int x, int d,
                                               const cpx<T>* tw, cpx<T>* P, cpx<T>* zball) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  cpx<T>* zb = zball + wib * padded_len(N);
  for (int t = threadIdx.x; t < N * NH; t += blockDim.x) P[t + ((t / NH) >> 5)] = in[t];
  __syncthreads();
  // 1. y axis inverse: the plane's columns in place
  tile_ffts<T, N, +1>(NH, tw, tw + kTwLen, [&](int p, int j) { return P + tpad(j, NH, p); },
                      [](int) { return true; });
  __syncthreads();
  // 2. rows: two Hermitian half rows A, B as the pencil A + i B; the inverse
  //    transform's real part is row A, its imaginary part row B
  if constexpr (group_rows<T, N>()) {
    group_c2r_pairs<T, N>(
        N / 2, 2 * NH, tw + kTwLen,
        [&](int pr, int k, cpx<T>& A, cpx<T>& B) {
          const cpx<T>* pa = P + tpad(2 * pr, NH, 0);
          A = pa[k];
          B = pa[NH + k];
        },
        [&](int pr, int) { return P + tpad(2 * pr, NH, 0); },
        [&](int pr, int j, T re, T im) {
          T* orow = out + ((size_t)x * N + 2 * pr) * N * 4 + d;
          orow[(size_t)j * 4] = re;
          orow[(size_t)(N + j) * 4] = im;
        });
  } else {
  for (int pr = wib; pr < N / 2; pr += (int)(blockDim.x >> 5)) {
    const cpx<T>* pa = P + tpad(2 * pr, NH, 0);   // rows 2 pr and 2 pr + 1 are adjacent
    const cpx<T>* pb = pa + NH;
    for (int k = lane; k < NH; k += 32) {
      cpx<T> A = pa[k], Bv = pb[k];
      if (k == 0 || k == N / 2) {
        A.y = T(0);
        Bv.y = T(0);
      }
      zb[zpad(k)] = cpx<T>{A.x - Bv.y, A.y + Bv.x};
      if (k > 0 && k < N / 2) zb[zpad(N - k)] = cpx<T>{A.x + Bv.y, -A.y + Bv.x};   // conj A + i conj B
    }
    __syncwarp();
    cpx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = zb[zpad(lane + 32 * m)];
    __syncwarp();
    warp_fft<T, E, +1>(v, lane, tw);
    // stage the two output rows (2N reals, padded per 32) in the warp's pencil,
    // whose N + N/32 complex slots hold exactly that
    T* ob = reinterpret_cast<T*>(zb);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      const int j = out_index(k1, E, lane);
      ob[zpad(j)] = v[k1].x;
      ob[zpad(N + j)] = v[k1].y;
    }
    __syncwarp();
    T* orow = out + ((size_t)x * N + 2 * pr) * N * 4 + d;
    for (int t = lane; t < 2 * N; t += 32) orow[(size_t)t * 4] = ob[zpad(t)];
    __syncwarp();
  }
  }
}

template <typename T, int E>
__global__ void __launch_bounds__(group_rows<T, 32 * E>() ? 512 : 1024) kwp_fwd(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb = tw + tw_len<T, E>();
  cpx<T>* P = zb + (group_rows<T, N>() ? 0 : (blockDim.x >> 5) * padded_len(N));
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.y];
  const int x = blockIdx.x;
  cpx<T>* out = r.T1 + (size_t)x * N * NH;
  if (r.phi_fixed)
    plane_fwd_body<T, E, unsigned long long>(static_cast<unsigned long long*>(r.phi) + (size_t)x * N * N, r.in_scale,
                                             out, tw, P, zb);
  else
    plane_fwd_body<T, E, T>(static_cast<T*>(r.phi) + (size_t)x * N * N, 1.0, out, tw, P, zb);
}

template <typename T, int E>
__global__ void __launch_bounds__(group_rows<T, 32 * E>() ? 512 : 1024) kwp_inv(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb = tw + tw_len<T, E>();
  cpx<T>* P = zb + (group_rows<T, N>() ? 0 : (blockDim.x >> 5) * padded_len(N));
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.z];
  const int x = blockIdx.x, d = blockIdx.y;
  const size_t S = (size_t)N * N * NH;
  plane_inv_body<T, E>(r.T2 + d * S + (size_t)x * N * NH, r.grad, x, d, tw, P, zb);
}

// Inverse plane kernel over all three gradient components of one x-plane
// (H <= 64): y-axis inverse of the three planes, then c2r of row pairs per
// component into per-warp staging rows, then whole (gx, gy, gz, 0) nodes
// written as 16-byte vectors.  Every node is written once, in full sectors
// (the per-component kernel writes each node's sector three times in part,
// which costs a DRAM read per sector once the nodes exceed L2).
template <typename T, int E> constexpr size_t plane3_smem_bytes(int nw) {
  if (group_rows<T, 32 * E>()) return ((size_t)tw_len<T, E>() + 3 * ((size_t)32 * E * (16 * E + 1) + E)) * sizeof(cpx<T>);
  return ((size_t)tw_len<T, E>() + (size_t)nw * padded_len(32 * E) + 3 * ((size_t)32 * E * (16 * E + 1) + E)) * sizeof(cpx<T>) +
         (size_t)nw * 3 * padded_len(64 * E) * sizeof(T);
}

template <typename T> __device__ __forceinline__ void store_node4(T* p, T a, T b, T c) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, 0.f);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2*>(p)[1] = make_double2(c, 0.0);
  }
}

template <typename T, int E>
__device__ __forceinline__ void plane_inv3_body(const cpx<T>* __restrict__ in, size_t S, T* __restrict__ out, int x,
                                                const cpx<T>* tw, cpx<T>* P, cpx<T>* zball, T* oball) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  constexpr int PL = N * NH + E;             // one padded plane
  constexpr int OL = padded_len(2 * N);      // one component's two staged rows, padded
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  cpx<T>* zb = zball + wib * padded_len(N);
  T* ob = oball + wib * 3 * OL;
  for (int d = 0; d < 3; ++d)
    for (int t = threadIdx.x; t < N * NH; t += blockDim.x) P[d * PL + t + ((t / NH) >> 5)] = in[d * S + t];
  __syncthreads();
  // 1. y axis inverse: the three planes' columns in place
  for (int d = 0; d < 3; ++d) {
    cpx<T>* Pd = P + d * PL;
    tile_ffts<T, N, +1>(NH, tw, tw + kTwLen, [&](int p, int j) { return Pd + tpad(j, NH, p); },
                        [](int) { return true; });
  }
  __syncthreads();
  if constexpr (group_rows<T, N>()) {
    // 2. rows: per component, the pencils A + i B of the row pairs, each
    //    pair's two output rows staged as reals in its own rows of the plane;
    //    then whole (gx, gy, gz, 0) nodes
    for (int d = 0; d < 3; ++d) {
      cpx<T>* Pd = P + d * PL;
      group_c2r_pairs<T, N>(
          N / 2, 2 * NH, tw + kTwLen,
          [&](int pr, int k, cpx<T>& A, cpx<T>& B) {
            const cpx<T>* pa = Pd + tpad(2 * pr, NH, 0);
            A = pa[k];
            B = pa[NH + k];
          },
          [&](int pr, int) { return Pd + tpad(2 * pr, NH, 0); },
          [&](int pr, int j, T re, T im) {
            T* ob = reinterpret_cast<T*>(Pd + tpad(2 * pr, NH, 0));
            ob[j] = re;
            ob[N + j] = im;
          });
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
      const int y = t / N, j = t - y * N;
      const int off = tpad(y & ~1, NH, 0);
      const int f = (y & 1) * N + j;
      store_node4<T>(out + (((size_t)x * N + y) * N + j) * 4, reinterpret_cast<const T*>(P + off)[f],
                     reinterpret_cast<const T*>(P + PL + off)[f], reinterpret_cast<const T*>(P + 2 * PL + off)[f]);
    }
  } else {
  // 2. rows: per component, the two Hermitian half rows A, B as the pencil
  //    A + i B (real part: row A, imaginary part: row B), staged; then the
  //    two rows of nodes
  for (int pr = wib; pr < N / 2; pr += nw) {
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      const cpx<T>* pa = P + d * PL + tpad(2 * pr, NH, 0);   // rows 2 pr and 2 pr + 1 are adjacent
      const cpx<T>* pb = pa + NH;
      for (int k = lane; k < NH; k += 32) {
        cpx<T> A = pa[k], Bv = pb[k];
        if (k == 0 || k == N / 2) {
          A.y = T(0);
          Bv.y = T(0);
        }
        zb[zpad(k)] = cpx<T>{A.x - Bv.y, A.y + Bv.x};
        if (k > 0 && k < N / 2) zb[zpad(N - k)] = cpx<T>{A.x + Bv.y, -A.y + Bv.x};   // conj A + i conj B
      }
      __syncwarp();
      cpx<T> v[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = zb[zpad(lane + 32 * m)];
      __syncwarp();
      warp_fft<T, E, +1>(v, lane, tw);
      T* obd = ob + d * OL;
#pragma unroll
      for (int k1 = 0; k1 < E; ++k1) {
        const int j = out_index(k1, E, lane);
        obd[zpad(j)] = v[k1].x;
        obd[zpad(N + j)] = v[k1].y;
      }
    }
    __syncwarp();
    T* orow = out + ((size_t)x * N + 2 * pr) * N * 4;
    for (int t = lane; t < 2 * N; t += 32) {
      const int q = zpad(t);
      store_node4<T>(orow + (size_t)t * 4, ob[q], ob[OL + q], ob[2 * OL + q]);
    }
    __syncwarp();
  }
  }
}

template <typename T, int E>
__global__ void __launch_bounds__(group_rows<T, 32 * E>() ? 512 : 1024) kwp_inv3(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb = tw + tw_len<T, E>();
  cpx<T>* P = zb + (group_rows<T, N>() ? 0 : (blockDim.x >> 5) * padded_len(N));
  T* ob = reinterpret_cast<T*>(P + 3 * ((size_t)N * NH + E));
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.y];
  const int x = blockIdx.x;
  const size_t S = (size_t)N * N * NH;
  plane_inv3_body<T, E>(r.T2 + (size_t)x * N * NH, S, r.grad, x, tw, P, zb, ob);
}

// ---------------------------------------------------------------------------
// Cluster plane kernels: one x-plane per cluster of CS CTAs (CS = 2 at
// H = 128, 4 at H = 256, where a whole plane does not fit one CTA's shared
// memory or would leave SMs idle).  Each CTA owns a contiguous range of the
// plane's H/2+1 columns for all H rows, so the y-axis FFTs are local; the
// rows are shared out through distributed shared memory:
//   forward: CTA r transforms rows [r H/CS, (r+1) H/CS) (two real rows per
//            complex warp FFT) and stores each output column into the shared
//            memory of the CTA that owns it; after a cluster barrier every
//            CTA transforms its columns along y and writes them;
//   inverse: every CTA loads its columns of one gradient component, does their
//            y-axis inverse, and after a cluster barrier its rows' c2r pull
//            the other columns from the peers' shared memory; a second
//            barrier keeps each CTA's columns alive until all peers are done.
// The arithmetic is that of the plane kernels (same warp FFT, same order), so
// the results are the same bits.
// ---------------------------------------------------------------------------
template <int N, int CS> struct ColSplit {
  static constexpr int NH = N / 2 + 1;
  static constexpr int CP = (NH + CS - 1) / CS;   // columns per CTA (the last one may hold fewer)
  static constexpr int LD = CP;                   // row stride of the column block (odd for CS = 2, 4)
  static __device__ __forceinline__ int first(int r) { return r * CP; }
  static __device__ __forceinline__ int count(int r) { return min(CP, NH - r * CP); }
};

template <typename T, int E, int CS> constexpr size_t cplane_smem_bytes(int nw) {
  // column block: H rows of CP plus one slot per 32 rows; one padded pencil per warp
  return ((size_t)32 * E * ColSplit<32 * E, CS>::LD + E + (size_t)nw * row_scratch<T, 32 * E>() + tw_len<T, E>()) *
         sizeof(cpx<T>);
}

template <typename T, int E, int CS, typename Tin>
__device__ __forceinline__ void cplane_fwd_body(Tin* __restrict__ in, double in_scale, cpx<T>* __restrict__ out,
                                                const cpx<T>* tw, cpx<T>* Q, cpx<T>* zball) {
  namespace cg = cooperative_groups;
  constexpr int N = 32 * E;
  using CSp = ColSplit<N, CS>;
  constexpr int NH = CSp::NH, LD = CSp::LD;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  cpx<T>* zb = zball + wib * padded_len(N);
  cpx<T>* peer[CS];
#pragma unroll
  for (int o = 0; o < CS; ++o) peer[o] = cluster.map_shared_rank(Q, o);
  // every CTA of the cluster is running before any stores into its shared memory
  cluster.sync();
  // 1. this CTA's rows (row pairs), results pushed to the owners' column blocks
  constexpr int PAIRS = N / 2 / CS;
  if constexpr (group_rows<T, N>()) {
    cpx<T>* zs = zball + wib * row_scratch<T, N>();
    group_r2c_pairs<T, N>(
        PAIRS, 0, tw + kTwLen,
        [&](int pr, int j, T& a, T& b) {
          const size_t ra = (size_t)(2 * (rank * PAIRS + pr)) * N + j, rb = ra + N;
          const Tin va = in[ra], vb = in[rb];
          in[ra] = Tin(0);
          in[rb] = Tin(0);
          if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value) {
            a = (T)((double)(long long)va * in_scale);
            b = (T)((double)(long long)vb * in_scale);
          } else {
            a = (T)va;
            b = (T)vb;
          }
        },
        [&](int, int g) { return zs + g * group_ps<N>(); },
        [&](int pr, int k, cpx<T> A, cpx<T> B) {
          const int row = 2 * (rank * PAIRS + pr), o = k / LD, kl = k - o * LD;
          cpx<T>* dst = peer[o];
          dst[tpad(row, LD, kl)] = A;
          dst[tpad(row + 1, LD, kl)] = B;
        });
  } else {
  for (int i = wib; i < PAIRS; i += nw) {
    const int pr = rank * PAIRS + i;
    const size_t ra = (size_t)(2 * pr) * N, rb = ra + N;
    cpx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const Tin a = in[ra + lane + 32 * m], b = in[rb + lane + 32 * m];
      if constexpr (sizeof(Tin) == 8 && !std::is_floating_point<Tin>::value)
        v[m] = cpx<T>{(T)((double)(long long)a * in_scale), (T)((double)(long long)b * in_scale)};
      else
        v[m] = cpx<T>{(T)a, (T)b};
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
      in[ra + lane + 32 * m] = Tin(0);
      in[rb + lane + 32 * m] = Tin(0);
    }
    warp_fft<T, E, -1>(v, lane, tw);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) zb[zpad(out_index(k1, E, lane))] = v[k1];
    __syncwarp();
    for (int k = lane; k < NH; k += 32) {
      const cpx<T> zk = zb[zpad(k)];
      const cpx<T> zm = cconj(zb[zpad((N - k) & (N - 1))]);
      const cpx<T> d = csub(zk, zm);
      const int o = k / LD, kl = k - o * LD;
      cpx<T>* dst = peer[o];
      dst[tpad(2 * pr, LD, kl)] = cpx<T>{(zk.x + zm.x) * T(0.5), (zk.y + zm.y) * T(0.5)};
      dst[tpad(2 * pr + 1, LD, kl)] = cpx<T>{d.y * T(0.5), -d.x * T(0.5)};
    }
    __syncwarp();
  }
  }
  cluster.sync();
  // 2. y axis of this CTA's columns
  const int c0 = CSp::first(rank), nc = CSp::count(rank);
  tile_ffts<T, N, -1>(nc, tw, tw + kTwLen, [&](int p, int j) { return Q + tpad(j, LD, p); },
                      [](int) { return true; });
  __syncthreads();
  for (int t = threadIdx.x; t < N * nc; t += blockDim.x) {
    const int j = t / nc, c = t - j * nc;
    out[(size_t)j * NH + c0 + c] = Q[tpad(j, LD, c)];
  }
}

template <typename T, int E, int CS>
__device__ __forceinline__ void cplane_inv_body(const cpx<T>* __restrict__ in, T* __restrict__ out, int x, int d,
                                                const cpx<T>* tw, cpx<T>* Q, cpx<T>* zball) {
  namespace cg = cooperative_groups;
  constexpr int N = 32 * E;
  using CSp = ColSplit<N, CS>;
  constexpr int NH = CSp::NH, LD = CSp::LD;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  cpx<T>* zb = zball + wib * padded_len(N);
  const int c0 = CSp::first(rank), nc = CSp::count(rank);
  for (int t = threadIdx.x; t < N * nc; t += blockDim.x) {
    const int j = t / nc, c = t - j * nc;
    Q[tpad(j, LD, c)] = in[(size_t)j * NH + c0 + c];
  }
  __syncthreads();
  // 1. y-axis inverse of this CTA's columns
  tile_ffts<T, N, +1>(nc, tw, tw + kTwLen, [&](int p, int j) { return Q + tpad(j, LD, p); },
                      [](int) { return true; });
  cluster.sync();
  const cpx<T>* peer[CS];
#pragma unroll
  for (int o = 0; o < CS; ++o) peer[o] = cluster.map_shared_rank(Q, o);
  // 2. this CTA's rows: two Hermitian half rows A, B as the pencil A + i B
  constexpr int PAIRS = N / 2 / CS;
  if constexpr (group_rows<T, N>()) {
    cpx<T>* zs = zball + wib * row_scratch<T, N>();
    group_c2r_pairs<T, N>(
        PAIRS, 0, tw + kTwLen,
        [&](int pr, int k, cpx<T>& A, cpx<T>& B) {
          const int row = 2 * (rank * PAIRS + pr), o = k / LD, kl = k - o * LD;
          A = peer[o][tpad(row, LD, kl)];
          B = peer[o][tpad(row + 1, LD, kl)];
        },
        [&](int, int g) { return zs + g * group_ps<N>(); },
        [&](int pr, int j, T re, T im) {
          T* orow = out + ((size_t)x * N + 2 * (rank * PAIRS + pr)) * N * 4 + d;
          orow[(size_t)j * 4] = re;
          orow[(size_t)(N + j) * 4] = im;
        });
  } else {
  for (int i = wib; i < PAIRS; i += nw) {
    const int pr = rank * PAIRS + i;
    for (int k = lane; k < NH; k += 32) {
      const int o = k / LD, kl = k - o * LD;
      cpx<T> A = peer[o][tpad(2 * pr, LD, kl)], Bv = peer[o][tpad(2 * pr + 1, LD, kl)];
      if (k == 0 || k == N / 2) {
        A.y = T(0);
        Bv.y = T(0);
      }
      zb[zpad(k)] = cpx<T>{A.x - Bv.y, A.y + Bv.x};
      if (k > 0 && k < N / 2) zb[zpad(N - k)] = cpx<T>{A.x + Bv.y, -A.y + Bv.x};
    }
    __syncwarp();
    cpx<T> v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = zb[zpad(lane + 32 * m)];
    __syncwarp();
    warp_fft<T, E, +1>(v, lane, tw);
    T* ob = reinterpret_cast<T*>(zb);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) {
      const int j = out_index(k1, E, lane);
      ob[zpad(j)] = v[k1].x;
      ob[zpad(N + j)] = v[k1].y;
    }
    __syncwarp();
    T* orow = out + ((size_t)x * N + 2 * pr) * N * 4 + d;
    for (int t = lane; t < 2 * N; t += 32) orow[(size_t)t * 4] = ob[zpad(t)];
    __syncwarp();
  }
  }
  // the peers may still read this CTA's columns
  cluster.sync();
}

template <typename T, int E, int CS>
__global__ void __launch_bounds__(1024) kwc_fwd(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb = tw + tw_len<T, E>();
  cpx<T>* Q = zb + (blockDim.x >> 5) * row_scratch<T, N>();
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.y];
  const int x = blockIdx.x / CS;
  cpx<T>* out = r.T1 + (size_t)x * N * NH;
  if (r.phi_fixed)
    cplane_fwd_body<T, E, CS, unsigned long long>(static_cast<unsigned long long*>(r.phi) + (size_t)x * N * N,
                                                  r.in_scale, out, tw, Q, zb);
  else
    cplane_fwd_body<T, E, CS, T>(static_cast<T*>(r.phi) + (size_t)x * N * N, 1.0, out, tw, Q, zb);
}

template <typename T, int E, int CS>
__global__ void __launch_bounds__(1024) kwc_inv(const FftRun<T>* __restrict__ runs) {
  constexpr int N = 32 * E, NH = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* zb = tw + tw_len<T, E>();
  cpx<T>* Q = zb + (blockDim.x >> 5) * row_scratch<T, N>();
  load_tw_group<T, E>(tw);
  __syncthreads();
  const FftRun<T>& r = runs[blockIdx.z];
  const int x = blockIdx.x / CS, d = blockIdx.y;
  const size_t S = (size_t)N * N * NH;
  cplane_inv_body<T, E, CS>(r.T2 + d * S + (size_t)x * N * NH, r.grad, x, d, tw, Q, zb);
}

// Launch with a cluster of CS CTAs along x.
template <typename K, typename... Args>
static cudaError_t launch_cluster(K kernel, dim3 grid, int threads, size_t smem, int cs, cudaStream_t s,
                                  Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

static int warp_blocks(int rows) {
  int b = (rows / 2 + 7) / 8;
  return b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b);
}

template <typename T, int E>
static cudaError_t warp_rows_r2c(const void* in, int in_kind, double in_scale, bool zero_input, cpx<T>* out, int rows,
                                 double* mass_acc, cudaStream_t s) {
  if (in_kind == 0)
    kw_rows_r2c<T, E, T><<<warp_blocks(rows), 256, 0, s>>>((T*)in, in_scale, zero_input ? 1 : 0, out, rows, mass_acc);
  else
    kw_rows_r2c<T, E, unsigned long long><<<warp_blocks(rows), 256, 0, s>>>((unsigned long long*)in, in_scale,
                                                                           zero_input ? 1 : 0, out, rows, mass_acc);
  return cudaGetLastError();
}

template <typename T, int E, int DIR>
static cudaError_t warp_cols(cpx<T>* data, int A, int B, int ncomp, size_t comp_stride, double scale, cudaStream_t s) {
  constexpr int BC = 16;
  const size_t smem = (tw_len<T, E>() + (size_t)32 * E * (BC + 1) + E) * sizeof(cpx<T>);
  auto k = kw_cols<T, E, DIR, BC>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((B + BC - 1) / BC, A, ncomp);
  k<<<grid, 256, smem, s>>>(data, B, comp_stride, (T)scale);
  return cudaGetLastError();
}

template <typename T, int E, int MODE>
static cudaError_t warp_spectral(const cpx<T>* T1, cpx<T>* alpha, cpx<T>* T2, SpecParams sp, double* shadow,
                                 cudaStream_t s) {
  constexpr int N = 32 * E;
  if constexpr (sizeof(T) == 4 && N <= 128) {
    constexpr int nw = 8;
    const size_t smem = xreg_smem_bytes<N>(nw);
    auto k = kwr_spectral_x<N, MODE>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(XRegShape<N>::TASKS + nw - 1) / nw, 32 * nw, smem, s>>>(T1, alpha, T2, sp, shadow);
    return cudaGetLastError();
  } else {
  constexpr int BC = (sizeof(T) == 8 && E == 8) ? 4 : ((sizeof(T) == 8 || E == 8) ? 8 : 16);
  const int B = N * (N / 2 + 1);
  const size_t smem = (kTwLen + twq_len<T, N>() + (size_t)N * (3 * BC + 1) + E) * sizeof(cpx<T>);
  auto k = kw_spectral_x<T, E, MODE, BC>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<(B + BC - 1) / BC, 256, smem, s>>>(T1, alpha, T2, sp, shadow);
  return cudaGetLastError();
  }
}

template <typename T, int E, int NCOMP>
static cudaError_t warp_rows_c2r(const cpx<T>* in, size_t comp_stride, T* out, int rows, double* max_acc,
                                 cudaStream_t s) {
  constexpr int NOUT = NCOMP == 3 ? 4 : 1;
  const size_t smem = row_c2r_smem<T, E, NOUT>();
  auto k = kw_rows_c2r<T, E, NCOMP>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<warp_blocks(rows), 256, smem, s>>>(in, comp_stride, out, rows, max_acc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

static int rows_per_pair_block(int H, size_t elem, bool with_out4) {
  // row pairs per block: up to 8, bounded so the shared buffers stay <= ~96 KB
  int rp = 8;
  auto bytes = [&](int r) {
    size_t b = (size_t)r * (H + 1) * 2 * elem;
    if (with_out4) b += (size_t)2 * r * H * 4 * elem;
    return b;
  };
  while (rp > 1 && bytes(rp) > 96 * 1024) rp >>= 1;
  return rp;
}

template <typename T>
cudaError_t launch_rows_r2c(const void* in, int in_kind, double in_scale, bool zero_input, cpx<T>* out,
                            int H, int rows, double* mass_acc, cudaStream_t s) {
  if (H == 32) return warp_rows_r2c<T, 1>(in, in_kind, in_scale, zero_input, out, rows, mass_acc, s);
  if (H == 64) return warp_rows_r2c<T, 2>(in, in_kind, in_scale, zero_input, out, rows, mass_acc, s);
  if (H == 128) return warp_rows_r2c<T, 4>(in, in_kind, in_scale, zero_input, out, rows, mass_acc, s);
  if (H == 256) return warp_rows_r2c<T, 8>(in, in_kind, in_scale, zero_input, out, rows, mass_acc, s);
  const int lgH = ilog2(H);
  const int RP = rows_per_pair_block(H, sizeof(T), false);
  const size_t smem = (kNmax / 2 + (size_t)RP * (H + 1)) * sizeof(cpx<T>);
  const int blocks = (rows + 2 * RP - 1) / (2 * RP);
  cudaError_t e;
  if (in_kind == 0) {
    auto k = k_rows_r2c<T, T>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<blocks, kThreads, smem, s>>>((T*)in, in_scale, zero_input ? 1 : 0, out, lgH, rows, RP, mass_acc);
  } else {
    auto k = k_rows_r2c<T, unsigned long long>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<blocks, kThreads, smem, s>>>((unsigned long long*)in, in_scale, zero_input ? 1 : 0, out, lgH, rows,
                                     RP, mass_acc);
  }
  return cudaGetLastError();
}

template <typename T>
static int col_chunk(int H, int slots) {
  // columns per block: power of two, shared buffer <= ~96 KB
  int bc = 32;
  while (bc > 1 && (size_t)H * slots * bc * sizeof(cpx<T>) > 96 * 1024) bc >>= 1;
  return bc;
}

template <typename T>
cudaError_t launch_cols(cpx<T>* data, int H, int A, int B, int ncomp, size_t comp_stride, int dir, double scale,
                        cudaStream_t s) {
  if (H == 32) return dir < 0 ? warp_cols<T, 1, -1>(data, A, B, ncomp, comp_stride, scale, s)
                              : warp_cols<T, 1, +1>(data, A, B, ncomp, comp_stride, scale, s);
  if (H == 64) return dir < 0 ? warp_cols<T, 2, -1>(data, A, B, ncomp, comp_stride, scale, s)
                              : warp_cols<T, 2, +1>(data, A, B, ncomp, comp_stride, scale, s);
  if (H == 128) return dir < 0 ? warp_cols<T, 4, -1>(data, A, B, ncomp, comp_stride, scale, s)
                               : warp_cols<T, 4, +1>(data, A, B, ncomp, comp_stride, scale, s);
  if (H == 256) return dir < 0 ? warp_cols<T, 8, -1>(data, A, B, ncomp, comp_stride, scale, s)
                               : warp_cols<T, 8, +1>(data, A, B, ncomp, comp_stride, scale, s);
  const int lgH = ilog2(H);
  int BC = col_chunk<T>(H, 1);
  if (BC > 16) BC = 16;
  const int lgBC = ilog2(BC);
  const size_t smem = (kNmax / 2 + (size_t)H * BC) * sizeof(cpx<T>);
  dim3 grid((B + BC - 1) / BC, A, ncomp);
  cudaError_t e;
  if (dir < 0) {
    auto k = k_cols<T, -1>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<grid, kThreads, smem, s>>>(data, lgH, B, lgBC, comp_stride, (T)scale);
  } else {
    auto k = k_cols<T, +1>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<grid, kThreads, smem, s>>>(data, lgH, B, lgBC, comp_stride, (T)scale);
  }
  return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t spectral_mode(const cpx<T>* T1, cpx<T>* alpha, cpx<T>* T2, int H, SpecParams sp,
                                 double* shadow, cudaStream_t s) {
  const int lgH = ilog2(H);
  int BC = col_chunk<T>(H, 4);
  if (BC > 16) BC = 16;
  const int lgBC = ilog2(BC);
  const int B = H * (H / 2 + 1);
  const size_t smem = (kNmax / 2 + (size_t)H * 4 * BC) * sizeof(cpx<T>);
  auto k = k_spectral_x<T, MODE>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<(B + BC - 1) / BC, kThreads, smem, s>>>(T1, alpha, T2, lgH, lgBC, sp, shadow);
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t warp_spectral_mode(const cpx<T>* T1, cpx<T>* alpha, cpx<T>* T2, SpecParams sp, int mode,
                                      double* shadow, cudaStream_t s) {
  switch (mode) {
    case kModeStep: return warp_spectral<T, E, kModeStep>(T1, alpha, T2, sp, shadow, s);
    case kModeDensity: return warp_spectral<T, E, kModeDensity>(T1, alpha, T2, sp, nullptr, s);
    case kModeField: return warp_spectral<T, E, kModeField>(T1, alpha, T2, sp, nullptr, s);
    case kModeGradOnly: return warp_spectral<T, E, kModeGradOnly>(T1, alpha, T2, sp, nullptr, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_spectral_x(const cpx<T>* T1, cpx<T>* alpha, cpx<T>* T2, int H, SpecParams sp, int mode,
                              double* alpha0_shadow, cudaStream_t s) {
  if (H == 32) return warp_spectral_mode<T, 1>(T1, alpha, T2, sp, mode, alpha0_shadow, s);
  if (H == 64) return warp_spectral_mode<T, 2>(T1, alpha, T2, sp, mode, alpha0_shadow, s);
  if (H == 128) return warp_spectral_mode<T, 4>(T1, alpha, T2, sp, mode, alpha0_shadow, s);
  if (H == 256) return warp_spectral_mode<T, 8>(T1, alpha, T2, sp, mode, alpha0_shadow, s);
  switch (mode) {
    case kModeStep: return spectral_mode<T, kModeStep>(T1, alpha, T2, H, sp, alpha0_shadow, s);
    case kModeDensity: return spectral_mode<T, kModeDensity>(T1, alpha, T2, H, sp, nullptr, s);
    case kModeField: return spectral_mode<T, kModeField>(T1, alpha, T2, H, sp, nullptr, s);
    case kModeGradOnly: return spectral_mode<T, kModeGradOnly>(T1, alpha, T2, H, sp, nullptr, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_rows_c2r(const cpx<T>* in, int ncomp, size_t comp_stride, T* out, int H, int rows,
                            double* max_acc, cudaStream_t s) {
  if (H == 32) return ncomp == 3 ? warp_rows_c2r<T, 1, 3>(in, comp_stride, out, rows, nullptr, s)
                                 : warp_rows_c2r<T, 1, 1>(in, comp_stride, out, rows, max_acc, s);
  if (H == 64) return ncomp == 3 ? warp_rows_c2r<T, 2, 3>(in, comp_stride, out, rows, nullptr, s)
                                 : warp_rows_c2r<T, 2, 1>(in, comp_stride, out, rows, max_acc, s);
  if (H == 128) return ncomp == 3 ? warp_rows_c2r<T, 4, 3>(in, comp_stride, out, rows, nullptr, s)
                                  : warp_rows_c2r<T, 4, 1>(in, comp_stride, out, rows, max_acc, s);
  if (H == 256) return ncomp == 3 ? warp_rows_c2r<T, 8, 3>(in, comp_stride, out, rows, nullptr, s)
                                  : warp_rows_c2r<T, 8, 1>(in, comp_stride, out, rows, max_acc, s);
  const int lgH = ilog2(H);
  const int RP = rows_per_pair_block(H, sizeof(T), true);
  const int NOUT = ncomp == 3 ? 4 : 1;
  const size_t smem = (kNmax / 2 + (size_t)RP * (H + 1)) * sizeof(cpx<T>) + (size_t)2 * RP * H * NOUT * sizeof(T);
  const int blocks = (rows + 2 * RP - 1) / (2 * RP);
  cudaError_t e;
  if (ncomp == 3) {
    auto k = k_rows_c2r<T, 3>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<blocks, kThreads, smem, s>>>(in, comp_stride, out, lgH, rows, RP, nullptr);
  } else {
    auto k = k_rows_c2r<T, 1>;
    if ((e = set_smem(k, smem)) != cudaSuccess) return e;
    k<<<blocks, kThreads, smem, s>>>(in, comp_stride, out, lgH, rows, RP, max_acc);
  }
  return cudaGetLastError();
}

constexpr size_t kMaxSmem = 227 * 1024;

template <typename T, int E, int BC>
static size_t cols_smem() {
  return (tw_len<T, E>() + (size_t)32 * E * (BC + 1) + E) * sizeof(cpx<T>);
}
template <typename T, int E, int SBC>
static size_t spectral_smem() {
  return (kTwLen + twq_len<T, 32 * E>() + (size_t)32 * E * (3 * SBC + 1) + E) * sizeof(cpx<T>);
}

template <typename T, int E, int DIR, int BC>
static cudaError_t kwb_cols_launch(const FftRun<T>* runs, int nruns, int ncomp, cudaStream_t s) {
  constexpr int N = 32 * E, NHH = N / 2 + 1;
  const size_t smc = cols_smem<T, E, BC>();
  if (smc > kMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = set_smem(kwb_cols<T, E, DIR, BC>, smc)) != cudaSuccess) return e;
  kwb_cols<T, E, DIR, BC><<<dim3((NHH + BC - 1) / BC, N, nruns * ncomp), 256, smc, s>>>(runs, ncomp);
  return cudaGetLastError();
}

template <typename T, int E, int DIR>
static cudaError_t kwb_cols_bc(const FftRun<T>* runs, int nruns, int ncomp, int bc, cudaStream_t s) {
  switch (bc) {
    case 8: return kwb_cols_launch<T, E, DIR, 8>(runs, nruns, ncomp, s);
    case 32: return kwb_cols_launch<T, E, DIR, 32>(runs, nruns, ncomp, s);
    default: return kwb_cols_launch<T, E, DIR, 16>(runs, nruns, ncomp, s);
  }
}

template <typename T, int E, int SBC>
static cudaError_t kwb_spectral_launch(const FftRun<T>* runs, int nruns, int nw, cudaStream_t s) {
  constexpr int N = 32 * E, NHH = N / 2 + 1;
  cudaError_t e;
  if constexpr (sizeof(T) == 4 && N <= 128) {
    const size_t smr = xreg_smem_bytes<N>(nw);
    if (smr > kMaxSmem) return cudaErrorInvalidValue;
    if ((e = set_smem(kwrb_spectral_x<N>, smr)) != cudaSuccess) return e;
    kwrb_spectral_x<N><<<dim3((XRegShape<N>::TASKS + nw - 1) / nw, nruns), 32 * nw, smr, s>>>(runs);
    return cudaGetLastError();
  } else {
    const size_t sms = spectral_smem<T, E, SBC>();
    if (sms > kMaxSmem) return cudaErrorInvalidValue;
    if ((e = set_smem(kwb_spectral_x<T, E, SBC>, sms)) != cudaSuccess) return e;
    kwb_spectral_x<T, E, SBC><<<dim3((N * NHH + SBC - 1) / SBC, nruns), 32 * nw, sms, s>>>(runs);
    return cudaGetLastError();
  }
}

// Default x-pass tile: as wide as shared memory comfortably allows.
template <typename T, int E> static int default_sbc() {
  return (sizeof(T) == 8 && E == 8) ? 4 : ((sizeof(T) == 8 || E == 8) ? 8 : 16);
}

template <typename T, int E>
static cudaError_t field_batch_e(const FftRun<T>* runs, int nruns, int stages, const FieldTune& tune,
                                 cudaStream_t s, int* launched) {
  int dummy = 0;
  int& nk = launched ? *launched : dummy;
  constexpr int N = 32 * E;
  cudaError_t e;
  const int rows_budget = 152 * (tune.rows_per_sm > 0 ? tune.rows_per_sm : 8);
  const int rblocks = max(1, min(rows_budget / max(nruns, 1), (N * N / 2 + 7) / 8));
  const int bc = tune.bc > 0 ? tune.bc : 16;
  const int sbc = tune.sbc > 0 ? tune.sbc : default_sbc<T, E>();
  // default plane warps: 8, or, for a kernel whose blocks fill the 152 SMs
  // less than `fill` times over, up to `most` (at most one warp per 4 plane
  // rows); measured at H = 128, one run: 32 for the forward kernel's 128
  // blocks, 16 for the inverse kernel's 384 (two blocks per SM)
  auto plane_warps = [&](int blocks, int fill, int most) {
    return tune.plane_nw > 0 ? tune.plane_nw
                             : (blocks <= fill * 152 ? max(kDefaultPlaneWarps, min(most, N / 4)) : kDefaultPlaneWarps);
  };
  // rows by group FFTs (at most 16 warps a block, no per-warp pencils): 16
  // warps for the forward and three-component kernels, 8 for the
  // per-component inverse (three of its blocks fit an SM)
  constexpr bool SP = group_rows<T, N>();
  const int fnw = plane_warps(nruns * N, 2, SP ? 16 : 32), inw = SP ? (tune.plane_nw > 0 ? tune.plane_nw : 8)
                                                                     : plane_warps(3 * nruns * N, 4, 16),
            i3nw = plane_warps(nruns * N, 2, SP ? 16 : 32);
  const int snw = tune.spec_nw > 0 ? tune.spec_nw : kDefaultSpectralWarps;
  const size_t fsm = plane_smem_bytes<T, E>(fnw), ism = plane_smem_bytes<T, E>(inw);
  const size_t i3sm = plane3_smem_bytes<T, E>(i3nw);
  // cluster plane kernels (CS = 2 at H <= 128, 4 at H = 256) when asked: at
  // H = 128 (one run) and H = 256 they measured slower than the plane kernels
  // and the pencil passes, so they are a tuning candidate, not a default
  constexpr int CS = E >= 8 ? 4 : 2;
  const int cnw = tune.plane_nw > 0 ? tune.plane_nw : (E >= 8 ? 8 : 16);
  const size_t csm = cplane_smem_bytes<T, E, CS>(cnw);
  const bool cluster_ok = E >= 2 && csm <= kMaxSmem;
  const bool clusters = cluster_ok && tune.plane_mode == 2;
  const bool planes = !clusters && tune.plane_mode == 0 && E <= 4 && fsm <= kMaxSmem && ism <= kMaxSmem;
  // all three components per inverse plane block: where asked, or by default
  // where the x-plane blocks fill the SMs four times over and two blocks fit
  // an SM (many runs: the gradient nodes then exceed L2)
  const bool inv3 = planes && E <= 2 &&
                    (tune.inv3 == 1 ? i3sm <= kMaxSmem
                                    : tune.inv3 == 0 && nruns * N >= 4 * 152 && 2 * i3sm <= kMaxSmem);
  if (stages & kFieldForward) {
    if (clusters) {
      if ((e = set_smem(kwc_fwd<T, E, CS>, csm)) != cudaSuccess) return e;
      if ((e = launch_cluster(kwc_fwd<T, E, CS>, dim3(N * CS, nruns), 32 * cnw, csm, CS, s, runs)) != cudaSuccess)
        return e;
      nk += 1;
    } else if (planes) {
      if ((e = set_smem(kwp_fwd<T, E>, fsm)) != cudaSuccess) return e;
      kwp_fwd<T, E><<<dim3(N, nruns), 32 * fnw, fsm, s>>>(runs);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      nk += 1;
    } else {
      kwb_rows_r2c<T, E><<<dim3(rblocks, nruns), 256, 0, s>>>(runs);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = kwb_cols_bc<T, E, -1>(runs, nruns, 1, bc, s)) != cudaSuccess) return e;
      nk += 2;
    }
  }
  if (stages & kFieldSpectral) {
    switch (sbc) {
      case 4: e = kwb_spectral_launch<T, E, 4>(runs, nruns, snw, s); break;
      case 8: e = kwb_spectral_launch<T, E, 8>(runs, nruns, snw, s); break;
      default: e = kwb_spectral_launch<T, E, 16>(runs, nruns, snw, s); break;
    }
    if (e != cudaSuccess) return e;
    nk += 1;
  }
  if ((stages & kFieldInverse) && clusters) {
    if ((e = set_smem(kwc_inv<T, E, CS>, csm)) != cudaSuccess) return e;
    if ((e = launch_cluster(kwc_inv<T, E, CS>, dim3(N * CS, 3, nruns), 32 * cnw, csm, CS, s, runs)) != cudaSuccess)
      return e;
    nk += 1;
  } else if ((stages & kFieldInverse) && inv3) {
    if constexpr (E <= 2) {
      if ((e = set_smem(kwp_inv3<T, E>, i3sm)) != cudaSuccess) return e;
      kwp_inv3<T, E><<<dim3(N, nruns), 32 * i3nw, i3sm, s>>>(runs);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      nk += 1;
    }
  } else if ((stages & kFieldInverse) && planes) {
    if ((e = set_smem(kwp_inv<T, E>, ism)) != cudaSuccess) return e;
    kwp_inv<T, E><<<dim3(N, 3, nruns), 32 * inw, ism, s>>>(runs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    nk += 1;
  } else if (stages & kFieldInverse) {
    if ((e = kwb_cols_bc<T, E, +1>(runs, nruns, 3, bc, s)) != cudaSuccess) return e;
    const size_t smr = row_c2r_smem<T, E, 4>();
    if ((e = set_smem(kwb_rows_c2r<T, E>, smr)) != cudaSuccess) return e;
    kwb_rows_c2r<T, E><<<dim3(rblocks, nruns), 256, smr, s>>>(runs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    nk += 2;
  }
  return cudaSuccess;
}

template <typename T, int E> static bool field_tune_valid_e(const FieldTune& t) {
  const int bc = t.bc > 0 ? t.bc : 16, sbc = t.sbc > 0 ? t.sbc : default_sbc<T, E>();
  size_t c = bc == 8 ? cols_smem<T, E, 8>() : bc == 32 ? cols_smem<T, E, 32>() : cols_smem<T, E, 16>();
  size_t x = sbc == 4 ? spectral_smem<T, E, 4>() : sbc == 8 ? spectral_smem<T, E, 8>() : spectral_smem<T, E, 16>();
  const bool pnw_ok =
      t.plane_nw == 0 || t.plane_nw == 8 || t.plane_nw == 16 || (!group_rows<T, 32 * E>() && t.plane_nw == 32);
  const bool snw_ok = t.spec_nw == 0 || t.spec_nw == 8 || t.spec_nw == 16;
  const int pnw = t.plane_nw > 0 ? t.plane_nw : kDefaultPlaneWarps;
  const bool inv3_ok = t.inv3 == 0 || t.inv3 == 2 ||
                       (t.inv3 == 1 && t.plane_mode == 0 && E <= 2 && plane3_smem_bytes<T, E>(pnw) <= kMaxSmem);
  return (bc == 8 || bc == 16 || bc == 32) && (sbc == 4 || sbc == 8 || sbc == 16) && c <= kMaxSmem &&
         x <= kMaxSmem && t.rows_per_sm >= 0 && t.rows_per_sm <= 32 &&
         (t.plane_mode == 0 || t.plane_mode == 1 ||
          (t.plane_mode == 2 && E >= 2 && cplane_smem_bytes<T, E, (E >= 8 ? 4 : 2)>(pnw) <= kMaxSmem)) &&
         pnw_ok && snw_ok && inv3_ok &&
         (t.plane_mode != 0 || E > 4 || plane_smem_bytes<T, E>(pnw) <= kMaxSmem);
}

template <typename T> FieldTune field_tune_default(int H) {
  FieldTune t;
  t.bc = 16;
  t.rows_per_sm = 8;
  t.plane_mode = 0;
  t.plane_nw = kDefaultPlaneWarps;
  t.spec_nw = kDefaultSpectralWarps;
  switch (H) {
    case 32: t.sbc = default_sbc<T, 1>(); break;
    case 64: t.sbc = default_sbc<T, 2>(); break;
    case 128: t.sbc = default_sbc<T, 4>(); break;
    default: t.sbc = default_sbc<T, 8>(); break;
  }
  return t;
}

template <typename T> bool field_tune_valid(int H, const FieldTune& t) {
  switch (H) {
    case 32: return field_tune_valid_e<T, 1>(t);
    case 64: return field_tune_valid_e<T, 2>(t);
    case 128: return field_tune_valid_e<T, 4>(t);
    case 256: return field_tune_valid_e<T, 8>(t);
  }
  return false;
}

template <typename T>
cudaError_t launch_field_batch(const FftRun<T>* runs, int nruns, int H, int stages, cudaStream_t s,
                               const FieldTune& tune, int* launched) {
  if (nruns <= 0) return cudaSuccess;
  switch (H) {
    case 32: return field_batch_e<T, 1>(runs, nruns, stages, tune, s, launched);
    case 64: return field_batch_e<T, 2>(runs, nruns, stages, tune, s, launched);
    case 128: return field_batch_e<T, 4>(runs, nruns, stages, tune, s, launched);
    case 256: return field_batch_e<T, 8>(runs, nruns, stages, tune, s, launched);
  }
  return cudaErrorInvalidValue;
}

#define SIPF_INST(T)                                                                                          \
  template cudaError_t launch_rows_r2c<T>(const void*, int, double, bool, cpx<T>*, int, int, double*,        \
                                          cudaStream_t);                                                    \
  template cudaError_t launch_cols<T>(cpx<T>*, int, int, int, int, size_t, int, double, cudaStream_t);       \
  template cudaError_t launch_spectral_x<T>(const cpx<T>*, cpx<T>*, cpx<T>*, int, SpecParams, int, double*,  \
                                            cudaStream_t);                                                  \
  template cudaError_t launch_rows_c2r<T>(const cpx<T>*, int, size_t, T*, int, int, double*, cudaStream_t);     \
  template cudaError_t launch_field_batch<T>(const FftRun<T>*, int, int, int, cudaStream_t, const FieldTune&, int*); \
  template bool field_tune_valid<T>(int, const FieldTune&);                                                   \
  template FieldTune field_tune_default<T>(int);
SIPF_INST(float)
SIPF_INST(double)
#undef SIPF_INST

}  // namespace sipf
