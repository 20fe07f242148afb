// Device-side building blocks of the SIPF-PIC step: complex type, Philox4x32-10
// noise, periodic wrap and the Gamma_2 / Gamma_4 particle-grid stencils.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sipf {

template <typename T> struct cpx { T x, y; };

__device__ __forceinline__ int ilog2_dev(int v) { return 31 - __clz(v); }   // v a power of two
__device__ __forceinline__ float t_floor(float v) { return floorf(v); }
__device__ __forceinline__ double t_floor(double v) { return ::floor(v); }
__device__ __forceinline__ float t_exp(float v) { return expf(v); }
__device__ __forceinline__ double t_exp(double v) { return ::exp(v); }
__device__ __forceinline__ bool t_finite(float v) { return isfinite(v); }
__device__ __forceinline__ bool t_finite(double v) { return isfinite(v); }

template <typename T> __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// Complex product with its roundings spelled out (one product rounded, the
// other fused into it), so every kernel that inlines it, whatever the
// compiler's contraction choices around it, gives the same bits: the FFT
// kernels of a run and of a batch, or of two launch shapes, agree exactly.
__device__ __forceinline__ float t_mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double t_mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float t_fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double t_fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T> __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {t_fma_rn(a.x, b.x, -t_mul_rn(a.y, b.y)), t_fma_rn(a.x, b.y, t_mul_rn(a.y, b.x))};
}
template <typename T> __device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of
//   (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2, c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0)
// with the key bumped by (W0, W1) between rounds.  Two counter blocks that
// share a key are run together so the key schedule is computed once.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ void philox_round(u32x4& c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
  const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
  c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
}

__device__ __forceinline__ void philox2blocks(u32x4& a, u32x4& b, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(a, k0, k1);
    philox_round(b, k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Six standard normals for particle p at step n (blocks 0 and 1 of the counter
// (p lo, p hi, n, block)); Box-Muller pairs (u0,u1), (u2,u3), (u4,u5) with
// u = (x + 1/2) 2^-32.  Double: libdevice-accurate log / sincos.
__device__ __forceinline__ void normals6(uint64_t seed, uint64_t p, uint32_t n, double z[6]) {
  u32x4 a{(uint32_t)p, (uint32_t)(p >> 32), n, 0u};
  u32x4 b{(uint32_t)p, (uint32_t)(p >> 32), n, 1u};
  philox2blocks(a, b, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
  const double two_m32 = 2.3283064365386963e-10;   // 2^-32
  const double two_pi = 6.283185307179586;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double u1 = ((double)w[2 * j] + 0.5) * two_m32;
    const double u2 = ((double)w[2 * j + 1] + 0.5) * two_m32;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(two_pi * u2, &s, &c);
    z[2 * j] = r * c;
    z[2 * j + 1] = r * s;
  }
}

// Float: the same uniforms built from the mantissa bits (no integer to float
// conversion).  unit23(x) = ((x >> 9) + 1/2) 2^-23 exactly; unit32 adds the
// low 9 bits, giving (x + 1/2) 2^-32 rounded once to float.  The radius uses
// unit32 (the tail of sqrt(-2 ln u) is sensitive to u), the angle unit23.
// lg2, sin and cos come from the hardware approximations; the angle is taken
// as 2 pi (u - 1/2) in [-pi, pi] (the accurate range of the sine unit), so
// cos/sin of 2 pi u are the negated values.
__device__ __forceinline__ float unit23(uint32_t x) {
  // 1 + m 2^-23 minus (1 - 2^-24): exact by Sterbenz
  return __int_as_float(0x3F800000u | (x >> 9)) - 0.99999994039535522f;
}
__device__ __forceinline__ float unit32(uint32_t x) {
  // (1 + r/512) - (1 + 255.5/512) = (r - 255.5)/512, exact; scaled by 2^-23
  const float lo = __int_as_float(0x3F800000u | ((x & 511u) << 14)) - 1.4990234375f;
  return fmaf(lo, 1.1920928955078125e-07f, unit23(x));
}

__device__ __forceinline__ void normals6(uint64_t seed, uint64_t p, uint32_t n, float z[6]) {
  u32x4 a{(uint32_t)p, (uint32_t)(p >> 32), n, 0u};
  u32x4 b{(uint32_t)p, (uint32_t)(p >> 32), n, 1u};
  philox2blocks(a, b, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
  const float two_pi = 6.28318530717958648f;
  const float ln2x2 = 1.3862943611198906f;          // 2 ln 2
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float u1 = unit32(w[2 * j]);
    const float u2 = unit23(w[2 * j + 1]);
    const float r2 = -ln2x2 * __log2f(u1);           // -2 ln u1 >= 0
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));  // sqrt(r2), 0 at r2 = 0
    float s, c;
    __sincosf(two_pi * (u2 - 0.5f), &s, &c);
    z[2 * j] = -r * c;
    z[2 * j + 1] = -r * s;
  }
}

// Four standard normals for particle p at step n from block 0 alone (the 2D
// move): the same values as the first four of normals6.
__device__ __forceinline__ void philox1block(u32x4& a, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(a, k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}
__device__ __forceinline__ void normals4(uint64_t seed, uint64_t p, uint32_t n, double z[4]) {
  u32x4 a{(uint32_t)p, (uint32_t)(p >> 32), n, 0u};
  philox1block(a, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
  const double two_m32 = 2.3283064365386963e-10;   // 2^-32
  const double two_pi = 6.283185307179586;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const double u1 = ((double)w[2 * j] + 0.5) * two_m32;
    const double u2 = ((double)w[2 * j + 1] + 0.5) * two_m32;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(two_pi * u2, &s, &c);
    z[2 * j] = r * c;
    z[2 * j + 1] = r * s;
  }
}
__device__ __forceinline__ void normals4(uint64_t seed, uint64_t p, uint32_t n, float z[4]) {
  u32x4 a{(uint32_t)p, (uint32_t)(p >> 32), n, 0u};
  philox1block(a, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
  const float two_pi = 6.28318530717958648f;
  const float ln2x2 = 1.3862943611198906f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float u1 = unit32(w[2 * j]);
    const float u2 = unit23(w[2 * j + 1]);
    const float r2 = -ln2x2 * __log2f(u1);
    const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
    float s, c;
    __sincosf(two_pi * (u2 - 0.5f), &s, &c);
    z[2 * j] = -r * c;
    z[2 * j + 1] = -r * s;
  }
}

// ---------------------------------------------------------------------------
// Geometry helpers.
// ---------------------------------------------------------------------------
template <typename T> struct Geo {
  T L, invL, half_L;   // box side, 1/L, L/2
  T inv_h;             // H / L
  int H, mask;         // H and H - 1 (H a power of two)
};

// Periodic wrap into [-L/2, L/2): x - L floor(x/L + 1/2), with the rounding
// edge cases pushed back inside.
template <typename T> __device__ __forceinline__ T wrap_coord(T x, const Geo<T>& g) {
  T y = x - g.L * t_floor(x * g.invL + T(0.5));
  if (y >= g.half_L) y -= g.L;
  if (y < -g.half_L) y += g.L;
  return y;
}

// cell = floor(H x / L), lambda = H x / L - cell.
__device__ __forceinline__ void cell_lambda_u(double u, int& cell, double& lam) {
  const double f = ::floor(u);
  cell = (int)f;
  lam = u - f;
}
// Float: floor through round-to-nearest of u - 1/2 with the 1.5 * 2^23 shift
// (plain FP32 adds, |u| < 2^22).  At an exact integer u the result may be
// (u - 1, lambda = 1) instead of (u, 0); the stencils are continuous across
// cell faces, so both give the same weights.
__device__ __forceinline__ void cell_lambda_u(float u, int& cell, float& lam) {
  const float magic = 12582912.0f;                  // 1.5 * 2^23
  const float t = (u - 0.5f) + magic;
  cell = __float_as_int(t) - 0x4B400000;
  lam = u - (t - magic);
}
template <typename T> __device__ __forceinline__ void cell_lambda(T x, const Geo<T>& g, int& cell, T& lam) {
  cell_lambda_u(x * g.inv_h, cell, lam);
}

// 1D factors of the stencils for one axis: index -1, 0, 1, 2 of Gamma_4 and
// the inner pair of Gamma_2.
template <typename T> struct Axis4 { T om, l0, l1, o2; };

template <typename T> __device__ __forceinline__ Axis4<T> axis4(T l) {
  Axis4<T> a;
  a.l0 = T(1) - l;
  a.l1 = l;
  const T c = l * (T(1) - l) * T(1.0 / 6.0);
  a.om = -(T(2) - l) * c;   // -(2 - l) l (1 - l) / 6     (index -1)
  a.o2 = -(T(1) + l) * c;   // -(1 + l)(1 - l) l / 6      (index  2)
  return a;
}

// Per-axis node indices of the four stencil layers (cell offsets -1, 0, 1, 2):
// ia[o] is the contribution of layer o on that axis to the flat node index.
// Global grid: ((c + o - 1) & mask) * stride.
__device__ __forceinline__ void axis_layers_global(int c, int mask, int stride, int ia[4]) {
#pragma unroll
  for (int o = 0; o < 4; ++o) ia[o] = ((c + o - 1) & mask) * stride;
}

// Visit the 32 nodes of Gamma_4 (Eq. (4ord)) with in-cell offsets lambda:
// fn(flat_index, w * F_gamma).  Inner nodes carry the trilinear weight times
// 1 + sum_k lambda_k (1 - lambda_k)/2; the outer node with index -1 or 2 on one
// axis carries that axis' cubic factor times the bilinear weight of the other
// two axes.  ix/iy/iz: per-axis layer indices (see axis_layers_global).
template <typename T, typename Fn>
__device__ __forceinline__ void gamma4_visit(const int ix[4], const int iy[4], const int iz[4], T lx, T ly, T lz,
                                             T w, Fn&& fn) {
  Axis4<T> ax = axis4(lx);
  const Axis4<T> ay = axis4(ly), az = axis4(lz);
  const T boost = T(1) + T(0.5) * (lx * ax.l0 + ly * ay.l0 + lz * az.l0);
  // fold the particle weight into the x-axis factors
  ax.l0 *= w;
  ax.l1 *= w;
  ax.om *= w;
  ax.o2 *= w;
  const T wx[2] = {ax.l0, ax.l1}, wy[2] = {ay.l0, ay.l1}, wz[2] = {az.l0, az.l1};
  T byz[2][2], bxz[2][2], bxy[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      byz[a][b] = wy[a] * wz[b];
      bxz[a][b] = wx[a] * wz[b];
      bxy[a][b] = wx[a] * wy[b];
    }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const T fa = wx[a] * boost;
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c) fn(ix[a + 1] + iy[b + 1] + iz[c + 1], fa * byz[b][c]);
  }
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      fn(ix[0] + iy[b + 1] + iz[c + 1], ax.om * byz[b][c]);
      fn(ix[3] + iy[b + 1] + iz[c + 1], ax.o2 * byz[b][c]);
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      fn(ix[a + 1] + iy[0] + iz[c + 1], ay.om * bxz[a][c]);
      fn(ix[a + 1] + iy[3] + iz[c + 1], ay.o2 * bxz[a][c]);
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      fn(ix[a + 1] + iy[b + 1] + iz[0], az.om * bxy[a][b]);
      fn(ix[a + 1] + iy[b + 1] + iz[3], az.o2 * bxy[a][b]);
    }
}

// The 8 nodes of Gamma_2 (Eq. (2ord)): trilinear weights; uses layers 1 and 2.
template <typename T, typename Fn>
__device__ __forceinline__ void gamma2_visit(const int ix[4], const int iy[4], const int iz[4], T lx, T ly, T lz,
                                             T w, Fn&& fn) {
  const T wx[2] = {(T(1) - lx) * w, lx * w}, wy[2] = {T(1) - ly, ly}, wz[2] = {T(1) - lz, lz};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T wab = wx[a] * wy[b];
#pragma unroll
      for (int c = 0; c < 2; ++c) fn(ix[a + 1] + iy[b + 1] + iz[c + 1], wab * wz[c]);
    }
}

template <typename T, typename Fn>
__device__ __forceinline__ void stencil_visit(int order, const int ix[4], const int iy[4], const int iz[4], T lx, T ly,
                                              T lz, T w, Fn&& fn) {
  if (order == 4) gamma4_visit<T>(ix, iy, iz, lx, ly, lz, w, fn);
  else gamma2_visit<T>(ix, iy, iz, lx, ly, lz, w, fn);
}

// Stencil of a particle on the global periodic grid.
template <typename T, typename Fn>
__device__ __forceinline__ void stencil_visit_global(int order, int cx, int cy, int cz, T lx, T ly, T lz, T w,
                                                     const Geo<T>& g, Fn&& fn) {
  int ix[4], iy[4], iz[4];
  axis_layers_global(cx, g.mask, g.H * g.H, ix);
  axis_layers_global(cy, g.mask, g.H, iy);
  axis_layers_global(cz, g.mask, 1, iz);
  stencil_visit<T>(order, ix, iy, iz, lx, ly, lz, w, fn);
}

// ---------------------------------------------------------------------------
// TMA bulk copies (global -> shared) completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Order earlier generic-proxy accesses of shared memory before later TMA writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bytes: multiple of 16; both addresses 16-byte aligned.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// L2 policy for data read or written once per step (the particle arrays):
// evicted first, so the grids the field solve and the gather reuse stay in L2.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// tma_load_1d with an L2 cache policy.
__device__ __forceinline__ void tma_load_1d_policy(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                   uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
// Hint: bring [p, p + bytes) into L2 (bytes: multiple of 16; p 16-byte aligned).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Wait for phase `parity` of the barrier; gives up after `limit` polls and
// returns false (the caller reports the timeout instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace sipf
