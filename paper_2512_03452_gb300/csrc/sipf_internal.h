// Host-side declarations shared by the translation units of libsipf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sipf_device.cuh"

namespace sipf {

constexpr int kNmax = 256;            // largest supported H
constexpr int kThreads = 256;         // block size of the grid kernels

// Spectral-kernel parameters (all in double; kernels round to T).
struct SpecParams {
  double L, inv_L3;      // box side and 1 / L^3 (the F_H normalisation)
  double tau, eps, k2;   // tau, eps, k^2
  double H0;             // filter scale (0: off)
  double beta0;          // M0 / L^3, source of the FP64 zero-mode shadow
  int propagator;        // SIPF_PROP_*
};

enum SpecMode { kModeStep = 0, kModeDensity = 1, kModeField = 2, kModeGradOnly = 3 };

// Per-device constant tables (twiddles); idempotent, thread-safe.
cudaError_t ensure_device_tables();

// ---- FFT / spectral launchers (fft_kernels.cu) --------------------------------
// rows r2c: `rows` real rows of length H (in) -> half-spectrum rows (out).
// in_kind: 0 = T, 1 = int64 fixed point scaled by in_scale.  zero_input
// clears the input after reading.  mass_acc (nullable) receives the FP64 sum.
template <typename T>
cudaError_t launch_rows_r2c(const void* in, int in_kind, double in_scale, bool zero_input,
                            cpx<T>* out, int H, int rows, double* mass_acc, cudaStream_t s);
// c2c along the middle axis of [A][H][B] complex arrays, ncomp arrays spaced
// comp_stride apart.  dir = -1 forward, +1 inverse.
template <typename T>
cudaError_t launch_cols(cpx<T>* data, int H, int A, int B, int ncomp, size_t comp_stride, int dir,
                        double scale, cudaStream_t s);
// x-axis pass fused with the spectral work (see SpecMode).
template <typename T>
cudaError_t launch_spectral_x(const cpx<T>* T1, cpx<T>* alpha, cpx<T>* T2, int H, SpecParams sp,
                              int mode, double* alpha0_shadow, cudaStream_t s);
// rows c2r of ncomp (1 or 3) half-spectrum arrays spaced comp_stride apart;
// ncomp == 3 writes interleaved 4-wide nodes (gx, gy, gz, 0), ncomp == 1 a
// plain real grid.  max_acc (nullable, ncomp == 1): FP64 max of the output.
template <typename T>
cudaError_t launch_rows_c2r(const cpx<T>* in, int ncomp, size_t comp_stride, T* out, int H,
                            int rows, double* max_acc, cudaStream_t s);

// ---- particle launchers (particle_kernels.cu) -----------------------------------
template <typename T>
struct MoveArgs {
  T* x; T* y; T* z;
  int64_t P;
  const T* grad4;        // H^3 nodes x 4 (gx, gy, gz, 0)
  void* phi;             // deposit target (T, or int64 fixed point)
  Geo<T> g;
  T s_noise;             // sqrt(mu tau) (half) or sqrt(2 mu tau) (plain)
  T chitau;              // chi * tau
  T w;                   // M0 / P, or 2^60 / P in fixed-point mode
  uint64_t seed;
  uint32_t n;            // step index used as the noise counter
  int p2g, g2p, split;
  int fixed;             // deposit into int64 fixed point
  int* err;              // sticky error word (bit 0: non-finite position)
};
template <typename T> cudaError_t launch_move_deposit(const MoveArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_deposit(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, T w, void* phi,
                           int order, int fixed, cudaStream_t s);
template <typename T>
cudaError_t launch_gather(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, const T* f,
                          int ncomp, int interleaved4, int order, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_noise(uint64_t seed, int64_t step, int64_t first, int64_t P, T* z, cudaStream_t s);
template <typename T>
cudaError_t launch_moments(const T* x, const T* y, const T* z, int64_t P, double* acc2, cudaStream_t s);
template <typename T>
cudaError_t launch_aos_to_soa(const double* aos, int64_t P, Geo<T> g, T* x, T* y, T* z, cudaStream_t s);
template <typename T>
cudaError_t launch_alpha_energy(const cpx<T>* alpha, int H, double* acc2, cudaStream_t s);

template <typename T> Geo<T> make_geo(double L, int H);

}  // namespace sipf
