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

// One run of a batch, as seen by the batched FFT kernels.
template <typename T>
struct FftRun {
  void* phi;          // deposit grid: T, or int64 fixed point (phi_fixed)
  int phi_fixed;
  double in_scale;    // fixed point -> mass
  cpx<T>* T1;         // forward intermediate
  cpx<T>* alpha;      // alpha^(n)
  cpx<T>* T2;         // three gradient spectra
  T* grad;            // 4 H^3 nodes (gx, gy, gz, 0)
  SpecParams sp;
  double* shadow;     // FP64 zero-mode shadow
};

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

// The whole field solve of a step (F_H of phi, update of alpha, gradient
// spectra, their inverse transforms) for `nruns` runs of the same H (32, 64,
// 128 or 256), the run table in device memory.  `stages` selects the forward
// transform (2 launches), the spectral pass (1) and the inverse transforms
// (2).  A single run's step uses the same kernels with a one-entry table, so
// a run computes the same bits alone or in a batch.
enum { kFieldForward = 1, kFieldSpectral = 2, kFieldInverse = 4, kFieldAll = 7 };
// Launch shapes of the field solve (0: default): the column tile of the y
// passes (8, 16 or 32 pencils per block), the column tile of the fused x pass
// (4, 8 or 16), the blocks per SM given to the row passes, and whether the two
// inner axes run as one plane kernel per direction or as separate pencil
// passes.  Results agree to rounding; they do not depend on the tile shapes.
struct FieldTune {
  int bc = 0, sbc = 0, rows_per_sm = 0;
  int plane_mode = 0;   // 0: plane kernels for the inner axes where they fit (H <= 128), 1: pencil passes,
                        // 2: cluster plane kernels (H >= 64; each x-plane over 2 or 4 blocks)
  int plane_nw = 0;     // warps per block of the plane kernels (8, 16, 32)
  int spec_nw = 0;      // warps per block of the fused x pass (8, 16)
  int inv3 = 0;         // inverse plane kernel: 0 by grid size, 1 one block per x-plane for all three
                        // gradient components (H <= 64), 2 one block per (component, x-plane)
};
template <typename T>
cudaError_t launch_field_batch(const FftRun<T>* runs, int nruns, int H, int stages, cudaStream_t s,
                               const FieldTune& tune = FieldTune{}, int* launched = nullptr);   // += kernels launched
template <typename T> bool field_tune_valid(int H, const FieldTune& t);
template <typename T> FieldTune field_tune_default(int H);   // the shapes used when a field is 0

// FP64 FMA throughput probe: blocks x 256 threads x 8 chains x iters FMAs.
cudaError_t launch_fp64_fma(int blocks, int iters, double* sink, cudaStream_t s);

// ---- adjoint launchers (adjoint_kernels.cu) ----------------------------------------
// One reverse step over all particles (see k_adj_step).
template <typename T>
struct AdjArgs {
  const T* x;          // X^{n-1}, P each, in the order of `id`
  const T* y;
  const T* z;
  const uint32_t* id;  // particle of each entry (NULL: entry p is particle p)
  const T* grad4;      // g^{n-1}: (gx, gy, gz, 0) per node, 4 H^3
  const T* phibar;     // transpose-of-deposit cotangent grid phibar^{n-1}, H^3
  const T* phibar4;    // its z-quads (phibar at z - 1 ... z + 2 per node, 4 H^3), read by the Gamma_4 kernel
  T* xb4;              // Xbar as (x, y, z, 0) per particle, 4 P (in: Xbar^n, out: Xbar^{n-1})
  T* gbar;             // H^3 interleaved (x, y, z, -) nodes (accumulated)
  double* acc;         // [0] += sum tau V.Xbar (dJ/dchi), [1] += dJ/ds terms
  Geo<T> g;
  T s_noise, chitau, tau, w_inv_h;
  uint64_t seed;
  uint32_t n;          // step index of the forward step being reversed
  int64_t P;
  int p2g, g2p, split;
};
template <typename T> cudaError_t launch_adj_step(const AdjArgs<T>& a, cudaStream_t s);
// phibar -> z-quads (4 H^3: phibar at z - 1, z, z + 1, z + 2 of each node)
template <typename T> cudaError_t launch_adj_quads(const T* phibar, T* quads, int H, cudaStream_t s);
// gbar nodes -> three planes of H^3 (and the nodes cleared)
template <typename T> cudaError_t launch_adj_planes(T* gbar4, T* planes, int64_t H3, cudaStream_t s);
// Xbar^N as (x, y, z, 0) per particle (xb4: 4 P) from X^N in particle order.
template <typename T>
cudaError_t launch_adj_terminal(const T* x, const T* y, const T* z, int64_t P, const T* phibar, int p2g, T w_inv_h,
                                Geo<T> g, T* xb4, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_spectral(const cpx<T>* ghat, cpx<T>* abar, cpx<T>* spec, int H, SpecParams sp, cudaStream_t s);

// ---- particle launchers (particle_kernels.cu) -----------------------------------
// One work item of the binned kernel: `len` particles of bin `bin` from slot `start`.
struct ChunkDesc {
  long long start;
  int bin, len;
};

// Arguments of the binned particle kernel (see particle_kernels.cu).
template <typename T>
struct BinArgs {
  // source bins
  const T* sx; const T* sy; const T* sz; const uint32_t* sid;
  const long long* src_base;     // [NT+1] first slot of each bin
  const int* src_count;          // [NT+1] particles in each bin
  const long long* chunk_start;  // [NT+2] prefix sum of ceil(count / chunk)
  const ChunkDesc* chunks;       // [chunk_start[NT+1]] work items
  // destination bins
  T* dx; T* dy; T* dz; uint32_t* did;
  const long long* dst_base;     // [NT+1]
  const int* dst_cap;            // [NT+1]
  int* dst_cursor;               // [NT+1] fill cursors (zeroed before the launch)
  unsigned long long* work;      // chunk counter of the persistent grid (zeroed before the launch)
  int NT, ntx, tile_shift;       // tiles, tiles per axis, log2 tile edge
  // physics
  void* phi;                     // deposit target (T, or int64 fixed point)
  const T* grad4;                // H^3 nodes x 4 (gx, gy, gz, 0)
  Geo<T> g;
  T s_noise;                     // sqrt(mu tau) (half) or sqrt(2 mu tau) (plain)
  T chitau;                      // chi * tau
  T wmass;                       // M0 / P
  int fix_k;                     // deterministic mode: fixed-point unit 2^-fix_k of a weight
  uint64_t seed;
  uint32_t n;                    // step index (noise counter)
  int p2g, g2p, split, fixed;
  int* err;                      // sticky error word: bit 0 non-finite position, bit 1 lost particle
};
// Per-run argument tables of the batched bookkeeping kernels.
struct ChunkListArgs {
  const int* cursor;        // fill cursors of the buffer just written
  const int* cap;
  const long long* base;
  int* count;
  long long* chunk_start;   // [NT+2]
  ChunkDesc* chunks;
  int* other_cursor;        // cursors of the other buffer (cleared)
  int NT;
  long long* part;          // chunk totals of the blocks of kCLBlock bins (chunk_list_blocks(NT))
  int merge;                // bins per merge window of the small bins (power of two, 2 ... 16)
};
struct LayoutArgs {
  const int* want;
  int* cap;
  long long* base;
  int NT, ntx, ovf_cap;
};
template <typename T>
cudaError_t launch_move_batch(const BinArgs<T>* table, const long long* prefix, int nruns, unsigned long long* work,
                              const uint32_t* step, bool move, cudaStream_t s, int blocks_per_sm = 0,
                              int g2p = 0);   // g2p: 2 or 4 when all runs use that gather order, else 0
template <typename T>
cudaError_t launch_deposit_batch(const BinArgs<T>* table, const long long* prefix, int nruns,
                                 unsigned long long* work, bool fixed, cudaStream_t s, int blocks_per_sm = 0);
cudaError_t launch_chunk_list_batch(const ChunkListArgs* t, int nruns, int max_NT, cudaStream_t s);
cudaError_t launch_run_prefix(const ChunkListArgs* t, int nruns, long long* prefix, unsigned long long* work,
                              uint32_t* step, int bump, cudaStream_t s);
cudaError_t launch_layout_batch(const LayoutArgs* t, int nruns, cudaStream_t s);
int binned_window_slots(int H);
int binned_chunk();
int binned_tile_shift(int H);
template <typename T> cudaError_t launch_binned(const BinArgs<T>& a, int move, int deposit, int rebin, cudaStream_t s);
// The move + re-bin pass of a step (Algorithm 4 particle loop).
template <typename T> cudaError_t launch_move(const BinArgs<T>& a, cudaStream_t s);
// From fill cursors: clamped counts, chunk prefix sums and chunk descriptors
// (slots from `base`); clears other_cursor and the work counter.  ovf_total
// (nullable) accumulates the number of particles in the overflow bin.
// Chunk list of one buffer: two launches (count, emit); clears work[0] and
// work[1] (a context's deposit / re-bin and move counters) and adds the
// overflow-bin count to *ovf_total when those are non-NULL.
int chunk_list_blocks(int NT);
cudaError_t launch_chunk_list(const ChunkListArgs& a, unsigned long long* work, unsigned long long* ovf_total,
                              cudaStream_t s);
cudaError_t launch_layout(const int* want, int* cap, long long* base, int NT, int ntx, int ovf_cap, cudaStream_t s);
template <typename T>
cudaError_t launch_tile_hist(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, int shift, int ntx, int NT,
                             int* hist, cudaStream_t s);
// Block-privatised re-bin of particle-order arrays; returns false (nothing
// launched) when there are too many tiles for a shared-memory count.
template <typename T>
bool launch_rebin_plain(const T* x, const T* y, const T* z, const uint32_t* id, int64_t P, Geo<T> g, int shift,
                        int ntx, int NT, T* dx, T* dy, T* dz, uint32_t* did, const long long* dst_base,
                        const int* dst_cap, int* dst_cursor, int* err, cudaStream_t s, cudaError_t* e,
                        int64_t id0 = 0,      // id == NULL: particle p gets id id0 + p
                        bool wrap = false);   // wrap the positions into the box as they are read
int rebin_plain_max_tiles();
// The two passes of launch_unbin with a scratch array, separately: binned
// particles to their ids' slots of the 4-wide scratch, and (any range of)
// the scratch to three arrays.
template <typename T> cudaError_t launch_unbin_aos(const BinArgs<T>& a, int64_t max_chunks, T* aos, cudaStream_t s);
template <typename T> cudaError_t launch_aos4_to_soa(const T* aos, int64_t P, T* x, T* y, T* z, cudaStream_t s);
// The current bins' particles into contiguous x, y, z, id (P each), grouped
// by work item in bin order (cursor: device scratch, cleared here).
template <typename T>
cudaError_t launch_compact(const BinArgs<T>& a, int64_t max_chunks, unsigned long long* cursor, T* x, T* y, T* z,
                           uint32_t* id, cudaStream_t s);
// Read-back in particle order by pieces of ids: np pieces, piece k holding ids
// [b[k], b[k+1]) (b[0] = 0, b[np] = P).
struct PieceBounds {
  static constexpr int kMax = 8;
  long long b[kMax + 1];
  int np;
};
// the current bins' particles as SoA records grouped by piece (piece k's at
// b[k] on); cursor: np ints, zeroed before the launch
template <typename T>
cudaError_t launch_partition_pieces(const BinArgs<T>& a, int64_t max_chunks, const PieceBounds& pb, int* cursor, T* rx,
                                    T* ry, T* rz, uint32_t* rid, cudaStream_t s);
// Particle order from the current bins through a slot map (slot_of: P
// entries, slots < 2^32): x[id] = X[slot_of[id]], written in id order; x, y, z
// may be host memory the device can address.
template <typename T>
cudaError_t launch_read_back_mapped(const BinArgs<T>& a, int64_t max_chunks, uint32_t* slot_of, int64_t P, T* x, T* y,
                                   T* z, cudaStream_t s);
// records [a0, a0 + n) scattered to x, y, z at their ids (ids >= P skipped)
template <typename T>
cudaError_t launch_scatter_piece(const T* rx, const T* ry, const T* rz, const uint32_t* rid, int64_t a0, int64_t n,
                                 int64_t P, T* x, T* y, T* z, cudaStream_t s);
template <typename T>
// Particle order from the bins; with aos_scratch (4 P elements) through a
// 4-wide scratch array and a transpose, else by three scattered stores.
cudaError_t launch_unbin(const BinArgs<T>& a, int64_t max_chunks, T* x, T* y, T* z, T* aos_scratch, int64_t P,
                         cudaStream_t s);
cudaError_t launch_iota(uint32_t* id, int64_t P, cudaStream_t s);
template <typename T>
cudaError_t launch_deposit(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, T w, T* phi, int order,
                           cudaStream_t s);
template <typename T>
cudaError_t launch_gather(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, const T* f, int ncomp, int order,
                          T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_noise(uint64_t seed, int64_t step, int64_t first, int64_t P, T* z, cudaStream_t s);
template <typename T>
cudaError_t launch_moments(const T* x, const T* y, const T* z, int64_t P, double* acc2, cudaStream_t s);
template <typename T>
cudaError_t launch_aos_to_soa(const double* aos, int64_t P, Geo<T> g, T* x, T* y, T* z, cudaStream_t s);
template <typename T> cudaError_t launch_wrap_soa(int64_t P, Geo<T> g, T* x, T* y, T* z, cudaStream_t s);
template <typename T>
cudaError_t launch_alpha_energy(const cpx<T>* alpha, int H, double* acc2, cudaStream_t s);

template <typename T> Geo<T> make_geo(double L, int H);

// Error reporting and parameter helpers of the C ABI (sipf_api.cu): set the
// calling thread's last error message and return the code.
int report_error(int code, const std::string& msg);
int report_cuda(cudaError_t e, const char* where);

}  // namespace sipf
