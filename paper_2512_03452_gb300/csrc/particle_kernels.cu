// Particle kernels of the SIPF-PIC step.
//
// Particles live in tile bins: the grid is cut into tiles of 8^3 cells and the
// particle arrays (x, y, z, id) are grouped by the tile of their cell, each bin
// with some spare capacity, plus an overflow bin; two such buffers alternate.
//   k_move:   the move of Algorithm 4 (noise keyed by the particle id, gather
//             of grad c with I* (Algorithm 3), drift, periodic wrap) for rounds
//             of a bin's particles staged in shared memory by bulk copies,
//             each particle then written into the bin of its new tile in the
//             other buffer (one global reservation per round and tile; the
//             particles of a merged item reserve one slot each);
//   chunk lists: work items of up to 4096 particles of one bin, and one
//             merged item per window of m consecutive bins for the bins
//             under 256 particles (m = 4 for a single run, 16 in a batch);
//   k_binned (deposit): the deposit I of the new positions (Algorithm 2), a
//             block per work item, into a shared-memory integer window over
//             the tile and the stencil halo (several copies, chosen per lane
//             so that a warp's atomics fall into distinct banks), then added
//             to the grid with coalesced reductions.  Particles outside the
//             window (the overflow bin) deposit with global reductions.
// Batched forms take the work items of many runs from one counter.  Also
// here: the re-binning of particle-order arrays, the read-backs to particle
// order (through a slot map, or by pieces of ids) and the bin-order copy of
// the positions that the adjoint's segments keep.
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

// ---------------------------------------------------------------------------
// Accumulation.  The shared-memory window holds integers (native shared
// atomics): int32 for float runs, int64 for double runs, in units of 2^-K of
// a stencil weight F.  In the default mode K is chosen per chunk so that no
// node sum can overflow (|F| <= 1, at most `len` particles per chunk), and the
// window is added to the floating-point grid as v * (M0/P) * 2^-K.  In the
// deterministic mode K is fixed for the run and the global grid is an int64
// fixed-point sum in the same units, so every addition is exact and the
// result does not depend on the order of the additions.
// ---------------------------------------------------------------------------
template <typename T> struct WinType;
template <> struct WinType<float> {
  using type = int;
  static constexpr int bits = 30;
  static __device__ __forceinline__ int round(float v) { return __float2int_rn(v); }
};
template <> struct WinType<double> {
  using type = long long;
  static constexpr int bits = 62;
  static __device__ __forceinline__ long long round(double v) { return __double2ll_rn(v); }
};

__device__ __forceinline__ int ceil_log2(int v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

// Most particles of a work item of `len` that can add into one copy of an
// int32 window, for blocks of `threads`.  Tile windows rank a warp's lanes
// within the G bank groups of their base slot and take copy = rank mod C
// (C copies, G = 32 / C groups), so one copy gets at most ceil(n_g / C) lanes
// of group g: at most sum_g ceil(n_g / C) <= (32 + G (C - 1)) / C of a warp
// (7 for C = 8, 14 for C = 4).  Whole-grid windows take copy = lane mod 4:
// 8 lanes of a warp.  Every particle adds at most once to a node with
// |round(F 2^K)| <= 2^K (|F| <= 1), so a copy's node sum stays within
// load * 2^K; K = 30 - ceil(log2(load + 1)) keeps it below 2^30.
__device__ __forceinline__ int win_copy_load(int per_warp, int len, int threads) {
  return per_warp * (threads >> 5) * ((len + threads - 1) / threads);
}

// 2^k from the exponent bits (no FP64 or transcendental call), |k| < 126
template <typename T> __device__ __forceinline__ T pow2(int k);
template <> __device__ __forceinline__ float pow2<float>(int k) { return __int_as_float((127 + k) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int k) {
  return __longlong_as_double((long long)(1023 + k) << 52);
}

// two's-complement integer adds into the shared window
__device__ __forceinline__ void win_add(int* p, int v) { atomicAdd(p, v); }
__device__ __forceinline__ void win_add(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
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

// Gather of the three gradient components (interleaved 4-wide nodes).
template <typename T>
__device__ __forceinline__ V3<T> gather_grad(const T* __restrict__ grad4, int order, T px, T py, T pz,
                                             const Geo<T>& g) {
  int cx, cy, cz;
  T lx, ly, lz;
  cell_lambda(px, g, cx, lx);
  cell_lambda(py, g, cy, ly);
  cell_lambda(pz, g, cz, lz);
  V3<T> acc{T(0), T(0), T(0)};
  stencil_visit_global<T>(order, cx, cy, cz, lx, ly, lz, T(1), g, [&](int idx, T f) {
    const V3<T> v = Vec4<T>::load(grad4 + (size_t)idx * 4);
    acc.x += f * v.x;
    acc.y += f * v.y;
    acc.z += f * v.z;
  });
  return acc;
}

__device__ __forceinline__ int tile_of(int cx, int cy, int cz, int shift, int ntx) {
  return (((cx >> shift) * ntx) + (cy >> shift)) * ntx + (cz >> shift);
}

// Find the run of global work item c: largest r with prefix[r] <= c.
__device__ __forceinline__ int find_run(const long long* prefix, int nruns, long long c) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// The binned particle kernel.  Template flags:
//   MOVE:    advance X^{n-1} -> X^n (Algorithm 4, particle loop)
//   DEPOSIT: deposit the positions into phi
//   REBIN:   write each particle into the destination bins of its tile
// A step runs MOVE+REBIN, then DEPOSIT over the new bins: the chemotactic
// drift can carry particles many cells in one step, so the deposit reads the
// bins of the new positions, where every particle lies in the tile of its bin
// and the window only needs the stencil halo.
// WHOLE: the window is the whole (small) grid with periodic slots (H <= 16);
// otherwise the window is the tile plus the halo of Gamma_4 (-1, +2).
// ---------------------------------------------------------------------------
constexpr int kTileShift = 3;                 // tiles of 8^3 cells
constexpr int kTileE = 1 << kTileShift;
constexpr int kMargin = 0;                    // deposits read bins of the current positions
constexpr int kWin = kTileE + 2 * kMargin + 3;  // 11 nodes per axis (tile + stencil halo)
constexpr int kWinSlots = kWin * kWin * kWin;
constexpr int kReplicas = 4;                  // whole-grid window copies (lane mod 4), one after another
// Tile windows keep kTileReps copies interleaved word by word (slot s, copy r
// at s * kTileReps + r; lane mod kTileReps picks the copy), so the lanes of a
// warp that share a copy hit banks that differ unless their slots agree mod
// 32 / kTileReps: far fewer bank conflicts than copies stored one after
// another, whose random slots spread over all 32 banks at random.
constexpr int kTileReps = 8;
constexpr int kChunk = 4096;                  // particles per work item
// Work items with fewer particles deposit with global reductions: clearing
// and flushing a tile window (11^3 slots x 8 copies) costs more than their
// 32 reductions per particle.
constexpr int kWinMinLen = 64;
// Sparse bins are taken together: the bins with fewer than kSmall particles
// (the overflow bin excepted) of each window of m consecutive bins form one
// work item, marked by bin = -m with the window index in `start` and the
// bins' total in `len`.  A sparse region then costs the move one round per
// window instead of one per bin.  m (a power of two, 2 ... kMergeMax) is set
// per chunk list: 4 for a single run (longer merged items left the deposit's
// last blocks idle), 16 for the runs of a batch (many sparse runs).
constexpr int kMergeMax = 16;
constexpr int kSmall = 256;
__device__ __forceinline__ int merge_of(const ChunkDesc& d) { return -d.bin; }
__device__ __forceinline__ bool bin_is_small(int b, int count, int NT) { return b < NT && count > 0 && count < kSmall; }

// Calls fn(slot) for every particle of work item d, the block's threads
// striding over each run of slots (all threads take the same bins).
template <typename T, typename Fn>
__device__ __forceinline__ void item_slots(const BinArgs<T>& a, const ChunkDesc& d, Fn&& fn) {
  if (d.bin >= 0) {
    for (int i = threadIdx.x; i < d.len; i += blockDim.x) fn(d.start + i);
    return;
  }
  const int m = merge_of(d);
  for (int k = 0; k < m; ++k) {
    const int b = (int)d.start * m + k;
    if (b > a.NT) break;
    const int c = a.src_count[b];
    if (!bin_is_small(b, c, a.NT)) continue;
    const long long s0 = a.src_base[b];
    for (int i = threadIdx.x; i < c; i += blockDim.x) fn(s0 + i);
  }
}

// Add the shared window (all replicas) to the grid and clear it; the
// reductions of a warp hit contiguous nodes along the fastest axis.  Tile
// windows of ints go 32 slots per warp pass in 16-byte pieces; whole-grid and
// 64-bit windows one slot per thread.  (ox, oy, oz): node of slot (0,0,0).
// A window node's 64-bit sum as T with one rounding.  Float: without a 64-bit
// integer conversion (which runs on the slow FP64 pipe): the copies of an
// int32 window sum to |v| < 2^34, so hi = v >> 16 and lo = v & 0xffff convert
// exactly from 32-bit integers, hi * 2^16 is exact, and the fused add rounds
// once.  Double (int64 windows): the plain conversion.
template <typename T> __device__ __forceinline__ T sum_to_real(long long v);
template <> __device__ __forceinline__ float sum_to_real<float>(long long v) {
  const int hi = (int)(v >> 16), lo = (int)(v & 0xffff);
  return __fmaf_rn((float)hi, 65536.0f, (float)lo);
}
template <> __device__ __forceinline__ double sum_to_real<double>(long long v) { return (double)v; }

template <typename T, bool FIXED, bool WHOLE>
__device__ __forceinline__ void window_flush(const BinArgs<T>& a, typename WinType<T>::type* win, int wslots, int ox,
                                             int oy, int oz, T wwin) {
  using A = typename WinType<T>::type;
  const int H = a.g.H, mask = a.g.mask;
  const T unit = a.wmass / wwin;   // M0/P * 2^-K
  if constexpr (!WHOLE && sizeof(A) == 4) {
    // Tile window of ints: a warp takes 32 consecutive slots (1 KB) per pass.
    // Lane l reads 16-byte pieces l and 32 + l (halves of slots l/2 and
    // 16 + l/2), the two halves of a slot are summed with the neighbour lane,
    // and lane l adds slot l/2 (even l) or 16 + l/2 (odd l) to the grid: 4
    // shared wavefronts per 512 bytes and a reduction from every lane.
    static_assert(kTileReps == 8, "two 16-byte halves per slot");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
    // (copies summed in 64 bits: a node's total over all copies may exceed 2^31)
    for (int s0 = warp * 32; s0 < wslots; s0 += nwarps * 32) {
      int4* base = reinterpret_cast<int4*>(win + (size_t)s0 * kTileReps);
      const int sa = s0 + (lane >> 1), sb = sa + 16;
      long long va = 0, vb = 0;
      if (sa < wslots) {
        const int4 q = base[lane];
        va = (long long)q.x + q.y + q.z + q.w;
        base[lane] = make_int4(0, 0, 0, 0);
      }
      if (sb < wslots) {
        const int4 q = base[32 + lane];
        vb = (long long)q.x + q.y + q.z + q.w;
        base[32 + lane] = make_int4(0, 0, 0, 0);
      }
      va += __shfl_xor_sync(0xFFFFFFFFu, va, 1);
      vb += __shfl_xor_sync(0xFFFFFFFFu, vb, 1);
      const int sidx = (lane & 1) ? sb : sa;
      const long long v = (lane & 1) ? vb : va;
      if (sidx < wslots && v != 0) {
        const int c = sidx % kWin, b = (sidx / kWin) % kWin, aa = sidx / (kWin * kWin);
        const int gi = (((ox + aa) & mask) * H + ((oy + b) & mask)) * H + ((oz + c) & mask);
        if (FIXED) atomicAdd(static_cast<unsigned long long*>(a.phi) + gi, (unsigned long long)(long long)v);
        else atomicAdd(static_cast<T*>(a.phi) + gi, sum_to_real<T>(v) * unit);
      }
    }
  } else {
    for (int sidx = threadIdx.x; sidx < wslots; sidx += blockDim.x) {
      long long v = 0;
      if (WHOLE) {
#pragma unroll
        for (int r = 0; r < kReplicas; ++r) {
          v += win[r * wslots + sidx];
          win[r * wslots + sidx] = A(0);
        }
      } else {
#pragma unroll
        for (int r = 0; r < kTileReps; ++r) {
          v += win[sidx * kTileReps + r];
          win[sidx * kTileReps + r] = A(0);
        }
      }
      if (v != 0) {
        int gi;
        if (WHOLE) {
          gi = sidx;
        } else {
          const int c = sidx % kWin, b = (sidx / kWin) % kWin, aa = sidx / (kWin * kWin);
          gi = (((ox + aa) & mask) * H + ((oy + b) & mask)) * H + ((oz + c) & mask);
        }
        if (FIXED) atomicAdd(static_cast<unsigned long long*>(a.phi) + gi, (unsigned long long)(long long)v);
        else atomicAdd(static_cast<T*>(a.phi) + gi, sum_to_real<T>(v) * unit);
      }
    }
  }
}

// One work item of k_binned (deposit and/or re-bin without a move).
// seg_cnt / seg_base (shared memory, nseg entries; NULL: the item is the
// contiguous slots start ... start + len - 1): the item's particles are the
// runs of seg_cnt[k] slots from seg_base[k], one after another.
template <typename T, bool FIXED, bool MOVE, bool DEPOSIT, bool REBIN, bool WHOLE>
__device__ __forceinline__ void binned_chunk(const BinArgs<T>& a, const ChunkDesc& cur,
                                             typename WinType<T>::type* win, const int* seg_cnt = nullptr,
                                             const long long* seg_base = nullptr, int nseg = 0) {
  using A = typename WinType<T>::type;
  const int H = a.g.H, mask = a.g.mask;
  const int wslots = WHOLE ? H * H * H : kWinSlots;
  const int lane = threadIdx.x & 31;
  // lanes of a warp that land in the same cell add into different copies
  A* const my_win = win + (lane & (kReplicas - 1)) * wslots;
  const int bin = cur.bin, len = cur.len;
  const long long start = cur.start;
  // window origin (node coordinates of slot (0,0,0))
  bool has_win = DEPOSIT && (WHOLE || (bin < a.NT && len >= kWinMinLen));
  int ox = 0, oy = 0, oz = 0;
  if (!WHOLE && bin < a.NT) {
    const int tz = bin % a.ntx, ty = (bin / a.ntx) % a.ntx, tx = bin / (a.ntx * a.ntx);
    ox = tx * kTileE - kMargin - 1;
    oy = ty * kTileE - kMargin - 1;
    oz = tz * kTileE - kMargin - 1;
  }
  // window scale 2^K: no copy's node sum can reach 2^30 (int32 windows; see
  // win_copy_load) or 2^62 (int64 windows: the whole chunk's sum)
  const int K = FIXED ? a.fix_k
                      : (sizeof(A) == 4 ? 30 - ceil_log2(win_copy_load(WHOLE ? 8 : 7, len, blockDim.x) + 1)
                                        : WinType<T>::bits - ceil_log2(len + 1));
  const T wwin = pow2<T>(K);
  const int iters = (len + blockDim.x - 1) / blockDim.x;
  // next particle's data is loaded one iteration ahead (streaming loads: the
  // particle arrays are read once per pass, the grids stay in L2)
  auto slot_of = [&](int i) -> long long {
    if (!seg_cnt) return start + i;
    int k = 0;
    while (k < nseg - 1 && i >= seg_cnt[k]) i -= seg_cnt[k++];
    return seg_base[k] + i;
  };
  T px = T(0), py = T(0), pz = T(0);
  uint32_t pid = 0;
  if ((int)threadIdx.x < len) {
    const long long s = slot_of(threadIdx.x);
    px = __ldcs(a.sx + s);
    py = __ldcs(a.sy + s);
    pz = __ldcs(a.sz + s);
    pid = __ldcs(a.sid + s);
  }
  for (int it = 0; it < iters; ++it) {
    const int i = it * blockDim.x + threadIdx.x;
    const bool valid = i < len;
    T x = px, y = py, z = pz;
    const uint32_t id = pid;
    if (i + (int)blockDim.x < len) {
      const long long s = slot_of(i + blockDim.x);
      px = __ldcs(a.sx + s);
      py = __ldcs(a.sy + s);
      pz = __ldcs(a.sz + s);
      pid = __ldcs(a.sid + s);
    }
    if (MOVE && valid) {
      T nz[6];
      normals6(a.seed, (uint64_t)id, a.n, nz);
      if (a.split == 0) {
        // Z = X + W^- + chi tau I*(grad c)(X + W^-),  X^n = Z + W^+
        const T yx = x + a.s_noise * nz[0], yy = y + a.s_noise * nz[1], yz = z + a.s_noise * nz[2];
        const V3<T> gr = gather_grad(a.grad4, a.g2p, yx, yy, yz, a.g);
        x = wrap_coord((yx + a.chitau * gr.x) + a.s_noise * nz[3], a.g);
        y = wrap_coord((yy + a.chitau * gr.y) + a.s_noise * nz[4], a.g);
        z = wrap_coord((yz + a.chitau * gr.z) + a.s_noise * nz[5], a.g);
      } else {
        // X^n = X + chi tau I*(grad c)(X) + W,  W ~ N(0, 2 mu tau I)
        const V3<T> gr = gather_grad(a.grad4, a.g2p, x, y, z, a.g);
        x = wrap_coord((x + a.chitau * gr.x) + a.s_noise * nz[0], a.g);
        y = wrap_coord((y + a.chitau * gr.y) + a.s_noise * nz[1], a.g);
        z = wrap_coord((z + a.chitau * gr.z) + a.s_noise * nz[2], a.g);
      }
      if (!(t_finite(x) && t_finite(y) && t_finite(z))) atomicOr(a.err, 1);
    }
    int cx = 0, cy = 0, cz = 0;
    T lx = T(0), ly = T(0), lz = T(0);
    cell_lambda(x, a.g, cx, lx);
    cell_lambda(y, a.g, cy, ly);
    cell_lambda(z, a.g, cz, lz);
    // reserve the destination slot first: the atomic's round trip overlaps the deposit
    int t = 0, rank = 0, leader = 0, b0 = 0;
    if (REBIN) {
      t = tile_of(cx & mask, cy & mask, cz & mask, a.tile_shift, a.ntx);
      const unsigned key = valid ? (unsigned)t : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
      leader = __ffs(peers) - 1;
      rank = __popc(peers & ((1u << lane) - 1u));
      if (valid && lane == leader) b0 = atomicAdd(a.dst_cursor + t, __popc(peers));
    }
    bool fits = DEPOSIT && valid && has_win;
    int sx = 0, sy = 0, sz = 0;
    if (!WHOLE && fits) {
      sx = (cx - 1 - ox) & mask;
      sy = (cy - 1 - oy) & mask;
      sz = (cz - 1 - oz) & mask;
      fits = sx <= kWin - 4 && sy <= kWin - 4 && sz <= kWin - 4;
    }
    // Copy of the tile window each lane adds into.  A slot's kTileReps copies
    // cover a fixed group of banks, and the group of every stencil node of a
    // particle is its base slot's group shifted by the same amount for all
    // lanes; so lanes whose base slots share a group are ranked and take
    // distinct copies (conflict-free while at most kTileReps share a group).
    int cpy = lane & (kTileReps - 1);
    if (DEPOSIT && !WHOLE) {
      constexpr int kGroups = 32 * 4 / (kTileReps * (int)sizeof(A));   // bank groups: 4 (int), 2 (long long)
      const int cls = fits ? ((((sx * kWin) + sy) * kWin + sz) & (kGroups - 1)) : kGroups;
      const unsigned m0 = __ballot_sync(0xFFFFFFFFu, cls & 1), m1 = __ballot_sync(0xFFFFFFFFu, cls & 2),
                     m2 = __ballot_sync(0xFFFFFFFFu, cls & 4);
      const unsigned peers = ((cls & 1) ? m0 : ~m0) & ((cls & 2) ? m1 : ~m1) & ((cls & 4) ? m2 : ~m2);
      cpy = __popc(peers & ((1u << lane) - 1u)) & (kTileReps - 1);
    }
    if (DEPOSIT && valid) {
      if (fits) {
        int ix[4], iy[4], iz[4];
        if (WHOLE) {
          axis_layers_global(cx, mask, H * H, ix);
          axis_layers_global(cy, mask, H, iy);
          axis_layers_global(cz, mask, 1, iz);
          stencil_visit<T>(a.p2g, ix, iy, iz, lx, ly, lz, wwin,
                           [&](int idx, T f) { win_add(my_win + idx, WinType<T>::round(f)); });
        } else {
          // base slot plus compile-time offsets of the 4x4x4 box (interleaved copies)
          A* wb = win + (((sx * kWin) + sy) * kWin + sz) * kTileReps + cpy;
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            ix[o] = o * (kWin * kWin * kTileReps);
            iy[o] = o * (kWin * kTileReps);
            iz[o] = o * kTileReps;
          }
          stencil_visit<T>(a.p2g, ix, iy, iz, lx, ly, lz, wwin,
                           [&](int idx, T f) { win_add(wb + idx, WinType<T>::round(f)); });
        }
      } else if (FIXED) {
        unsigned long long* grid = static_cast<unsigned long long*>(a.phi);
        stencil_visit_global<T>(a.p2g, cx, cy, cz, lx, ly, lz, wwin, a.g, [&](int idx, T f) {
          atomicAdd(grid + idx, (unsigned long long)(long long)WinType<T>::round(f));
        });
      } else {
        T* grid = static_cast<T*>(a.phi);
        stencil_visit_global<T>(a.p2g, cx, cy, cz, lx, ly, lz, a.wmass, a.g,
                                [&](int idx, T f) { atomicAdd(grid + idx, f); });
      }
    }
    if (REBIN) {
      b0 = __shfl_sync(0xFFFFFFFFu, b0, leader);
      if (valid) {
        long long slot;
        const int r = b0 + rank;
        if (r < a.dst_cap[t]) {
          slot = a.dst_base[t] + r;
        } else {
          const int o = atomicAdd(a.dst_cursor + a.NT, 1);
          slot = o < a.dst_cap[a.NT] ? a.dst_base[a.NT] + o : -1;
        }
        if (slot >= 0) {
          a.dx[slot] = x;
          a.dy[slot] = y;
          a.dz[slot] = z;
          a.did[slot] = id;
        } else {
          atomicOr(a.err, 2);   // overflow bin full: the particle is lost
        }
      }
    }
  }
  if (DEPOSIT && has_win) {
    __syncthreads();
    window_flush<T, FIXED, WHOLE>(a, win, wslots, ox, oy, oz, wwin);
  }
}

// A work item of k_binned: one bin's chunk, or a merged item: its bins under
// kWinMinLen particles in one pass without a window, then each other small
// bin with its own window.
template <typename T, bool FIXED, bool MOVE, bool DEPOSIT, bool REBIN, bool WHOLE>
__device__ __forceinline__ void binned_item(const BinArgs<T>& a, const ChunkDesc& cur,
                                            typename WinType<T>::type* win) {
  if (cur.bin >= 0) {
    binned_chunk<T, FIXED, MOVE, DEPOSIT, REBIN, WHOLE>(a, cur, win);
    return;
  }
  // the window's bins, looked up together
  const int m = merge_of(cur);
  __shared__ int s_cnt[kMergeMax], s_tiny[kMergeMax];
  __shared__ long long s_base[kMergeMax];
  if (threadIdx.x < m) {
    const int b = (int)cur.start * m + threadIdx.x;
    int c = b <= a.NT ? a.src_count[b] : 0;
    if (!bin_is_small(b, c, a.NT)) c = 0;
    s_cnt[threadIdx.x] = c;
    s_tiny[threadIdx.x] = !WHOLE && c < kWinMinLen ? c : 0;
    s_base[threadIdx.x] = c ? a.src_base[b] : 0;
  }
  __syncthreads();
  // bins too small for a window: all of them in one pass (global reductions)
  int tiny = 0;
  for (int k = 0; k < m; ++k) tiny += s_tiny[k];
  if (tiny > 0)
    binned_chunk<T, FIXED, MOVE, DEPOSIT, REBIN, WHOLE>(a, ChunkDesc{0, a.NT, tiny}, win, s_tiny, s_base, m);
  // the others each with its window
  for (int k = 0; k < m; ++k) {
    const int c = s_cnt[k];
    if (c == 0 || s_tiny[k] != 0) continue;
    binned_chunk<T, FIXED, MOVE, DEPOSIT, REBIN, WHOLE>(a, ChunkDesc{s_base[k], (int)cur.start * m + k, c}, win);
    __syncthreads();   // the window's flush (which clears it) ends before the next bin adds into it
  }
}

template <typename T, bool FIXED, bool MOVE, bool DEPOSIT, bool REBIN, bool WHOLE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_binned(BinArgs<T> a) {
  using A = typename WinType<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* win = reinterpret_cast<A*>(smem_raw);
  __shared__ ChunkDesc s_desc[2];
  const long long nchunks = a.chunk_start[a.NT + 1];
  const int wslots = WHOLE ? a.g.H * a.g.H * a.g.H : kWinSlots;
  if (DEPOSIT)
    for (int i = threadIdx.x; i < (WHOLE ? kReplicas : kTileReps) * wslots; i += blockDim.x) win[i] = A(0);
  // work items are taken from a global counter; the next one is fetched
  // while the current one is processed
  if (threadIdx.x == 0) {
    const long long c = (long long)atomicAdd(a.work, 1ULL);
    s_desc[0] = c < nchunks ? a.chunks[c] : ChunkDesc{0, 0, 0};
  }
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const ChunkDesc cur = s_desc[buf];
    if (cur.len == 0) break;
    ChunkDesc nxt{0, 0, 0};
    if (threadIdx.x == 0) {
      const long long c = (long long)atomicAdd(a.work, 1ULL);
      if (c < nchunks) nxt = a.chunks[c];
    }
    binned_item<T, FIXED, MOVE, DEPOSIT, REBIN, WHOLE>(a, cur, win);
    if (threadIdx.x == 0) s_desc[buf ^ 1] = nxt;
    __syncthreads();
  }
}

// Batched deposit over the bins of all runs (tile windows, H >= 32).
template <typename T, bool FIXED>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
k_deposit_batch(const BinArgs<T>* __restrict__ table, const long long* __restrict__ prefix, int nruns,
                unsigned long long* work) {
  using A = typename WinType<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* win = reinterpret_cast<A*>(smem_raw);
  __shared__ ChunkDesc s_desc[2];
  __shared__ int s_run[2];
  const long long total = prefix[nruns];
  for (int i = threadIdx.x; i < kTileReps * kWinSlots; i += blockDim.x) win[i] = A(0);
  if (threadIdx.x == 0) {
    const long long c = (long long)atomicAdd(work, 1ULL);
    if (c < total) {
      const int r = find_run(prefix, nruns, c);
      s_run[0] = r;
      s_desc[0] = table[r].chunks[c - prefix[r]];
    } else {
      s_desc[0] = ChunkDesc{0, 0, 0};
    }
  }
  __syncthreads();
  for (int buf = 0;; buf ^= 1) {
    const ChunkDesc cur = s_desc[buf];
    if (cur.len == 0) break;
    const int run = s_run[buf];
    ChunkDesc nxt{0, 0, 0};
    int nrun = 0;
    if (threadIdx.x == 0) {
      const long long c = (long long)atomicAdd(work, 1ULL);
      if (c < total) {
        nrun = find_run(prefix, nruns, c);
        nxt = table[nrun].chunks[c - prefix[nrun]];
      }
    }
    binned_item<T, FIXED, false, true, false, false>(table[run], cur, win);
    if (threadIdx.x == 0) {
      s_desc[buf ^ 1] = nxt;
      s_run[buf ^ 1] = nrun;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Move + re-bin (the particle loop of Algorithm 4).  A block takes a work item
// (particles of one tile bin) in rounds of kMoveRound particles:
//   1. move each particle, stage (x, y, z, id) in shared memory and count its
//      destination tile among the 5^3 tiles around the source tile (shared
//      atomics hand out the rank inside that destination);
//   2. reserve each destination's range with one global atomic per tile;
//   3. write the staged particles to their slots.
// Destinations further than two tiles away (and particles of the overflow
// bin) reserve their slot with their own global atomic.  One global atomic
// per (round, destination tile) keeps dense tiles' cursors uncontended.
// ---------------------------------------------------------------------------
constexpr int kNbr = 125;   // 5^3 destination tiles around the source tile

constexpr int kMoveThreads = 256;   // threads per move block
template <typename T> struct MoveRound { static constexpr int n = (sizeof(T) == 4 ? 8 : 4) * kMoveThreads; };
template <typename T> constexpr int move_min_blocks() { return sizeof(T) == 4 ? 3 : 2; }

template <typename T>
struct MoveSmem {
  static constexpr int R = MoveRound<T>::n;
  ChunkDesc desc[2];
  int run[2];
  __align__(16) T x[R];
  __align__(16) T y[R];
  __align__(16) T z[R];
  __align__(16) uint32_t id[R];
  int meta[R];        // neighbour slot (0..124) | rank << 7, or -1 - tile for far moves
  int cnt[kNbr], base[kNbr], tile[kNbr], cap[kNbr];
  long long gbase[kNbr];   // first slot of each destination bin
  long long seg_base[kMergeMax];   // merged items: first slot and particles of each small bin
  int seg_cnt[kMergeMax];
  __align__(8) uint64_t bar;
  int abort;
};

// The move of one particle (Algorithm 4, particle loop): noise keyed by the
// id and step n, gather of grad c with I*, drift, periodic wrap.
template <typename T, int G2P>
__device__ __forceinline__ void move_one(const BinArgs<T>& a, uint32_t n, uint32_t id, T& x, T& y, T& z) {
  T nz[6];
  normals6(a.seed, (uint64_t)id, n, nz);
  if (a.split == 0) {
    // Z = X + W^- + chi tau I*(grad c)(X + W^-),  X^n = Z + W^+
    const T yx = x + a.s_noise * nz[0], yy = y + a.s_noise * nz[1], yz = z + a.s_noise * nz[2];
    const V3<T> gr = gather_grad(a.grad4, G2P ? G2P : a.g2p, yx, yy, yz, a.g);
    x = wrap_coord((yx + a.chitau * gr.x) + a.s_noise * nz[3], a.g);
    y = wrap_coord((yy + a.chitau * gr.y) + a.s_noise * nz[4], a.g);
    z = wrap_coord((yz + a.chitau * gr.z) + a.s_noise * nz[5], a.g);
  } else {
    // X^n = X + chi tau I*(grad c)(X) + W,  W ~ N(0, 2 mu tau I)
    const V3<T> gr = gather_grad(a.grad4, G2P ? G2P : a.g2p, x, y, z, a.g);
    x = wrap_coord((x + a.chitau * gr.x) + a.s_noise * nz[0], a.g);
    y = wrap_coord((y + a.chitau * gr.y) + a.s_noise * nz[1], a.g);
    z = wrap_coord((z + a.chitau * gr.z) + a.s_noise * nz[2], a.g);
  }
  if (!(t_finite(x) && t_finite(y) && t_finite(z))) atomicOr(a.err, 1);
}

// Tile of a position.
template <typename T> __device__ __forceinline__ int tile_of_pos(const BinArgs<T>& a, T x, T y, T z) {
  int cx, cy, cz;
  T l;
  cell_lambda(x, a.g, cx, l);
  cell_lambda(y, a.g, cy, l);
  cell_lambda(z, a.g, cz, l);
  const int mask = a.g.mask;
  return tile_of(cx & mask, cy & mask, cz & mask, a.tile_shift, a.ntx);
}

// Step 3 of a round: the staged particles written to their slots (meta: a
// neighbour slot with the rank inside its reservation, or -1 - tile for a
// particle that reserves its own slot).
template <typename T> __device__ __forceinline__ void move_write_out(const BinArgs<T>& a, MoveSmem<T>& sm, int cnt) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int meta = sm.meta[i];
    int r, cap;
    long long gb;
    if (meta >= 0) {
      const int k = meta & 127;
      r = sm.base[k] + (meta >> 7);
      cap = sm.cap[k];
      gb = sm.gbase[k];
    } else {
      const int t = -1 - meta;
      r = atomicAdd(a.dst_cursor + t, 1);
      cap = a.dst_cap[t];
      gb = a.dst_base[t];
    }
    long long slot;
    if (r < cap) {
      slot = gb + r;
    } else {
      const int o = atomicAdd(a.dst_cursor + a.NT, 1);
      slot = o < a.dst_cap[a.NT] ? a.dst_base[a.NT] + o : -1;
    }
    if (slot >= 0) {   // streaming stores (evicted from L2 first)
      __stcs(a.dx + slot, sm.x[i]);
      __stcs(a.dy + slot, sm.y[i]);
      __stcs(a.dz + slot, sm.z[i]);
      __stcs(a.did + slot, sm.id[i]);
    } else {
      atomicOr(a.err, 2);   // overflow bin full: the particle is lost
    }
  }
}

// A merged work item (small bins of one window): its particles, from several
// source tiles, are read straight from their bins in rounds, moved, staged
// and written out, each reserving its own destination slot (sparse bins, so
// the destination cursors see little contention).
template <typename T, bool MOVE, int G2P>
__device__ __forceinline__ void move_merged(const BinArgs<T>& a, const ChunkDesc& cur, uint32_t n, MoveSmem<T>& sm) {
  constexpr int R = MoveRound<T>::n;
  const int m = merge_of(cur);
  if (threadIdx.x < m) {
    const int b = (int)cur.start * m + threadIdx.x;
    int c = 0;
    long long base = 0;
    if (b <= a.NT) {
      c = a.src_count[b];
      base = a.src_base[b];
      if (!bin_is_small(b, c, a.NT)) c = 0;
    }
    sm.seg_cnt[threadIdx.x] = c;
    sm.seg_base[threadIdx.x] = base;
  }
  __syncthreads();
  for (int r0 = 0; r0 < cur.len; r0 += R) {
    const int cnt = min(R, cur.len - r0);
#pragma unroll 1
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      // the bin holding item particle r0 + i
      int k = 0, o = r0 + i;
      while (k < m - 1 && o >= sm.seg_cnt[k]) o -= sm.seg_cnt[k++];
      const long long slot = sm.seg_base[k] + o;
      T x = a.sx[slot], y = a.sy[slot], z = a.sz[slot];
      const uint32_t id = a.sid[slot];
      if (MOVE) move_one<T, G2P>(a, n, id, x, y, z);
      sm.x[i] = x;
      sm.y[i] = y;
      sm.z[i] = z;
      sm.id[i] = id;
      sm.meta[i] = -1 - tile_of_pos(a, x, y, z);
    }
    __syncthreads();
    move_write_out(a, sm, cnt);
    __syncthreads();
  }
}

// Warm L2 with the next round's particle arrays (x, y, z, id from slot s0,
// cnt particles; slots 4-aligned, bins padded to 4) while the current round
// is moved, so its bulk copies into shared memory do not wait on DRAM.
template <typename T>
__device__ __forceinline__ void prefetch_round(const BinArgs<T>& a, long long s0, int cnt) {
  const uint32_t n4 = (uint32_t)((cnt + 3) & ~3);
  l2_prefetch(a.sx + s0, n4 * sizeof(T));
  l2_prefetch(a.sy + s0, n4 * sizeof(T));
  l2_prefetch(a.sz + s0, n4 * sizeof(T));
  l2_prefetch(a.sid + s0, n4 * 4);
}

// One work item of the move + re-bin pass (see above).  n: step index of the
// move (noise counter).  MOVE = false only re-bins (capacity rebuilds).
// nxt / na (thread 0; na nullable): the block's next work item and its run's
// arguments, whose first round is prefetched during this item's last round.
template <typename T, bool MOVE, int G2P = 0>
__device__ __forceinline__ void move_chunk(const BinArgs<T>& a, const ChunkDesc& cur, uint32_t n, MoveSmem<T>& sm,
                                           uint32_t& phase, const ChunkDesc& nxt, const BinArgs<T>* na) {
  if (cur.bin < 0) {
    move_merged<T, MOVE, G2P>(a, cur, n, sm);
    return;
  }
  constexpr int R = MoveRound<T>::n;
  constexpr int PER = R / kMoveThreads;
  const int mask = a.g.mask, ntx = a.ntx, tmask = a.ntx - 1;   // tiles per axis: a power of two
  const bool in_tile = cur.bin < a.NT;
  const int stz = cur.bin & tmask, sty = (cur.bin / ntx) & tmask, stx = cur.bin / (ntx * ntx);
  // destination tile of each neighbour slot (periodic)
  for (int k = threadIdx.x; k < kNbr; k += blockDim.x) {
    const int dx = k / 25 - 2, dy = (k / 5) % 5 - 2, dz = k % 5 - 2;
    sm.tile[k] = ((((stx + dx) & tmask) * ntx) + ((sty + dy) & tmask)) * ntx + ((stz + dz) & tmask);
  }
  for (int r0 = 0; r0 < cur.len; r0 += R) {
    const int cnt = min(R, cur.len - r0);
    // stage the round's particles with TMA (bins start on 4-slot boundaries
    // and have capacity rounded up to 4, so the rounded copy stays inside)
    if (threadIdx.x == 0) {
      const long long s0 = cur.start + r0;
      const uint32_t n4 = (uint32_t)((cnt + 3) & ~3);
      fence_proxy_async_smem();
      mbar_expect_tx(&sm.bar, n4 * (3 * (uint32_t)sizeof(T) + 4));
      const uint64_t pol = l2_policy_evict_first();
      tma_load_1d_policy(sm.x, a.sx + s0, n4 * sizeof(T), &sm.bar, pol);
      tma_load_1d_policy(sm.y, a.sy + s0, n4 * sizeof(T), &sm.bar, pol);
      tma_load_1d_policy(sm.z, a.sz + s0, n4 * sizeof(T), &sm.bar, pol);
      tma_load_1d_policy(sm.id, a.sid + s0, n4 * 4, &sm.bar, pol);
      if (r0 + R < cur.len) prefetch_round(a, s0 + R, min(R, cur.len - r0 - R));
    }
    for (int k = threadIdx.x; k < kNbr; k += blockDim.x) sm.cnt[k] = 0;
    if (!mbar_wait(&sm.bar, phase, 1u << 26)) {
      atomicOr(a.err, 4);   // staging copy did not complete
      sm.abort = 1;
    }
    phase ^= 1;
    __syncthreads();
    if (sm.abort) return;
    // 1. move and stage
#pragma unroll 1
    for (int k = 0; k < PER; ++k) {
      const int i = k * kMoveThreads + threadIdx.x;
      if (i >= cnt) break;
      T x = sm.x[i], y = sm.y[i], z = sm.z[i];
      if (MOVE) move_one<T, G2P>(a, n, sm.id[i], x, y, z);
      int cx, cy, cz;
      T l;
      cell_lambda(x, a.g, cx, l);
      cell_lambda(y, a.g, cy, l);
      cell_lambda(z, a.g, cz, l);
      const int ux = (cx & mask) >> a.tile_shift, uy = (cy & mask) >> a.tile_shift, uz = (cz & mask) >> a.tile_shift;
      // destination relative to the source tile, minimum image in tile units
      const int half = ntx >> 1;
      const int dx = ((ux - stx + half) & tmask) - half;
      const int dy = ((uy - sty + half) & tmask) - half;
      const int dz = ((uz - stz + half) & tmask) - half;
      int meta;
      if (in_tile && dx >= -2 && dx <= 2 && dy >= -2 && dy <= 2 && dz >= -2 && dz <= 2) {
        const int nb = ((dx + 2) * 5 + (dy + 2)) * 5 + (dz + 2);
        meta = nb | (atomicAdd(sm.cnt + nb, 1) << 7);
      } else {
        meta = -1 - ((ux * ntx + uy) * ntx + uz);
      }
      sm.x[i] = x;
      sm.y[i] = y;
      sm.z[i] = z;
      sm.meta[i] = meta;
    }
    __syncthreads();
    // (the next item's descriptor has arrived by now)
    if (threadIdx.x == 0 && r0 + R >= cur.len && nxt.len > 0 && nxt.bin >= 0 && na)
      prefetch_round(*na, nxt.start, min(R, nxt.len));
    // 2. one reservation per destination tile (with its capacity and first slot)
    for (int k = threadIdx.x; k < kNbr; k += blockDim.x) {
      const int c = sm.cnt[k];
      if (c) {
        const int t = sm.tile[k];
        sm.base[k] = atomicAdd(a.dst_cursor + t, c);
        sm.cap[k] = a.dst_cap[t];
        sm.gbase[k] = a.dst_base[t];
      }
    }
    __syncthreads();
    // 3. write out
    move_write_out(a, sm, cnt);
    __syncthreads();
  }
}

template <typename T, int G2P>
__global__ void __launch_bounds__(kMoveThreads, move_min_blocks<T>())
k_move(BinArgs<T> a) {
  __shared__ MoveSmem<T> sm;
  const long long nchunks = a.chunk_start[a.NT + 1];
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    sm.abort = 0;
    const long long c = (long long)atomicAdd(a.work, 1ULL);
    sm.desc[0] = c < nchunks ? a.chunks[c] : ChunkDesc{0, 0, 0};
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int buf = 0;; buf ^= 1) {
    const ChunkDesc cur = sm.desc[buf];
    if (cur.len == 0 || sm.abort) break;
    ChunkDesc nxt{0, 0, 0};
    if (threadIdx.x == 0) {
      const long long c = (long long)atomicAdd(a.work, 1ULL);
      if (c < nchunks) nxt = a.chunks[c];
    }
    move_chunk<T, true, G2P>(a, cur, a.n, sm, phase, nxt, &a);
    if (threadIdx.x == 0) sm.desc[buf ^ 1] = nxt;
    __syncthreads();
  }
}


// Batched move (MOVE) or re-bin (!MOVE): work items of all runs from one
// counter; run r's arguments at table[r]; the step index from device memory.
template <typename T, bool MOVE, int G2P>
__global__ void __launch_bounds__(kMoveThreads, move_min_blocks<T>())
k_move_batch(const BinArgs<T>* __restrict__ table, const long long* __restrict__ prefix, int nruns,
             unsigned long long* work, const uint32_t* step) {
  __shared__ MoveSmem<T> sm;
  const long long total = prefix[nruns];
  const uint32_t n = *step + 1;
  if (threadIdx.x == 0) {
    mbar_init(&sm.bar, 1);
    sm.abort = 0;
    const long long c = (long long)atomicAdd(work, 1ULL);
    if (c < total) {
      const int r = find_run(prefix, nruns, c);
      sm.run[0] = r;
      sm.desc[0] = table[r].chunks[c - prefix[r]];
    } else {
      sm.desc[0] = ChunkDesc{0, 0, 0};
    }
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int buf = 0;; buf ^= 1) {
    const ChunkDesc cur = sm.desc[buf];
    if (cur.len == 0 || sm.abort) break;
    const int run = sm.run[buf];
    ChunkDesc nxt{0, 0, 0};
    int nrun = 0;
    if (threadIdx.x == 0) {
      const long long c = (long long)atomicAdd(work, 1ULL);
      if (c < total) {
        nrun = find_run(prefix, nruns, c);
        nxt = table[nrun].chunks[c - prefix[nrun]];
      }
    }
    move_chunk<T, MOVE, G2P>(table[run], cur, n, sm, phase, nxt, nxt.len > 0 ? table + nrun : nullptr);
    if (threadIdx.x == 0) {
      sm.desc[buf ^ 1] = nxt;
      sm.run[buf ^ 1] = nrun;
    }
    __syncthreads();
  }
}

template <typename T> cudaError_t launch_move(const BinArgs<T>& a, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  auto k = a.g2p == 4 ? k_move<T, 4> : k_move<T, 2>;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMoveThreads, 0)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k<<<sms * per_sm, kMoveThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe (the FP64 form's ALU bound): eight independent
// dependency chains per thread, `iters` fused multiply-adds each; the result
// is stored only if it is never reached, so nothing is optimised away.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* sink) {
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = (double)(threadIdx.x + k) * 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = fma(v[k], a, b);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  if (t == 12345.678) *sink = t;
}

cudaError_t launch_fp64_fma(int blocks, int iters, double* sink, cudaStream_t s) {
  k_fp64_fma<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-7, sink);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bin bookkeeping.
// ---------------------------------------------------------------------------
// From the fill cursors of the buffer just written: valid counts (clamped to
// capacity), the chunk prefix sum, the chunk descriptors, and the reset of the
// other buffer's cursors and of the work counter.  Two passes over blocks of
// kCLBlock bins: count (block-local exclusive prefix of chunks and the block
// total), then emit (block offset from the totals of the blocks before it,
// the descriptors, the grand total).
// ---------------------------------------------------------------------------
constexpr int kCLBlock = 1024;

__device__ __forceinline__ long long block_exclusive_scan_ll(long long v, long long& total) {
  __shared__ long long s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_w[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < nw ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    s_w[lane] = w;   // inclusive prefix of warp totals
  }
  __syncthreads();
  total = s_w[nw - 1];
  const long long ex = (wid > 0 ? s_w[wid - 1] : 0) + incl - v;
  __syncthreads();
  return ex;
}

__device__ __forceinline__ void chunk_count_body(const ChunkListArgs& a, int blk) {
  const int nb = a.NT + 1;
  const int b = blk * kCLBlock + threadIdx.x;
  long long ch = 0;
  bool small = false;
  if (b < nb) {
    const int c = min(a.cursor[b], a.cap[b]);
    a.count[b] = c;
    small = bin_is_small(b, c, a.NT);
    ch = small ? 0 : (c + kChunk - 1) / kChunk;
    a.other_cursor[b] = 0;
  }
  // the first bin of a window (a.merge lanes of a warp) also holds the
  // window's merged item, if it has small bins
  const unsigned sm = __ballot_sync(0xFFFFFFFFu, small);
  const int lane = threadIdx.x & 31, mw = a.merge;
  if ((lane & (mw - 1)) == 0 && ((sm >> lane) & ((1u << mw) - 1u)) != 0u) ch += 1;
  long long total;
  const long long ex = block_exclusive_scan_ll(ch, total);
  if (b < nb) a.chunk_start[b] = ex;
  if (threadIdx.x == 0) a.part[blk] = total;
}

__device__ __forceinline__ void chunk_emit_body(const ChunkListArgs& a, int blk, int nblk, unsigned long long* work,
                                                unsigned long long* ovf_total) {
  __shared__ long long s_off;
  __shared__ long long s_ls[kCLBlock];   // block-local first chunk of each bin
  if (threadIdx.x == 0) {
    long long o = 0;
    for (int i = 0; i < blk; ++i) o += a.part[i];
    s_off = o;
  }
  const long long total = a.part[blk];
  __syncthreads();
  const long long off = s_off;
  const int nb = a.NT + 1;
  const int b = blk * kCLBlock + threadIdx.x;
  if (b < nb) {
    const long long ls = a.chunk_start[b];
    a.chunk_start[b] = ls + off;
    s_ls[threadIdx.x] = ls;
  } else {
    s_ls[threadIdx.x] = total;
  }
  __syncthreads();
  // descriptors: one per thread, each finding its bin (the last bin whose first chunk is <= q)
  for (long long q = threadIdx.x; q < total; q += blockDim.x) {
    int i = 0;
#pragma unroll
    for (int step = kCLBlock / 2; step > 0; step >>= 1)
      if (s_ls[i + step] <= q) i += step;
    const int bin = blk * kCLBlock + i;
    int j = (int)(q - s_ls[i]);
    if ((bin & (a.merge - 1)) == 0) {
      int tot = 0;
      for (int k = 0; k < a.merge && bin + k < nb; ++k) {
        const int cc = a.count[bin + k];
        if (bin_is_small(bin + k, cc, a.NT)) tot += cc;
      }
      if (tot > 0) {
        if (j == 0) {   // the window's merged item comes first
          a.chunks[off + q] = ChunkDesc{(long long)(bin / a.merge), -a.merge, tot};
          continue;
        }
        j -= 1;
      }
    }
    const int c = a.count[bin];
    a.chunks[off + q] = ChunkDesc{a.base[bin] + (long long)j * kChunk, bin, min(kChunk, c - j * kChunk)};
  }
  if (blk == nblk - 1 && threadIdx.x == 0) {
    a.chunk_start[nb] = off + total;
    if (work) {   // a context's two work counters (deposit / re-bin, move)
      work[0] = 0ULL;
      work[1] = 0ULL;
    }
    if (ovf_total) *ovf_total += (unsigned long long)a.count[a.NT];
  }
}

__device__ __forceinline__ int chunk_list_blocks_dev(int NT) { return (NT + 1 + kCLBlock - 1) / kCLBlock; }

__global__ void __launch_bounds__(kCLBlock) k_chunk_count(ChunkListArgs a) { chunk_count_body(a, blockIdx.x); }

__global__ void __launch_bounds__(kCLBlock)
k_chunk_emit(ChunkListArgs a, unsigned long long* work, unsigned long long* ovf_total) {
  chunk_emit_body(a, blockIdx.x, gridDim.x, work, ovf_total);
}

// Batched: grid (blocks of the largest run, runs).
__global__ void __launch_bounds__(kCLBlock) k_chunk_count_batch(const ChunkListArgs* __restrict__ t) {
  const ChunkListArgs a = t[blockIdx.y];
  if ((int)blockIdx.x >= chunk_list_blocks_dev(a.NT)) return;
  chunk_count_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(kCLBlock) k_chunk_emit_batch(const ChunkListArgs* __restrict__ t) {
  const ChunkListArgs a = t[blockIdx.y];
  const int nblk = chunk_list_blocks_dev(a.NT);
  if ((int)blockIdx.x >= nblk) return;
  chunk_emit_body(a, blockIdx.x, nblk, nullptr, nullptr);
}

// Prefix over runs of their work-item counts; clears the work counter and,
// if asked, advances the batch's step counter.
__global__ void __launch_bounds__(1024)
k_run_prefix(const ChunkListArgs* __restrict__ t, int nruns, long long* __restrict__ prefix, unsigned long long* work,
             uint32_t* step, int bump) {
  __shared__ long long s_part[1024];
  const int per = (nruns + blockDim.x - 1) / blockDim.x;
  const int r0 = threadIdx.x * per;
  long long local = 0;
  for (int r = r0; r < min(r0 + per, nruns); ++r) local += t[r].chunk_start[t[r].NT + 1];
  s_part[threadIdx.x] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const long long v = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = s_part[threadIdx.x] - local;
  for (int r = r0; r < min(r0 + per, nruns); ++r) {
    prefix[r] = run;
    run += t[r].chunk_start[t[r].NT + 1];
  }
  if (threadIdx.x == blockDim.x - 1) prefix[nruns] = s_part[threadIdx.x];
  if (threadIdx.x == 0) {
    *work = 0ULL;
    if (bump) *step += 1u;
  }
}

// Capacities from the wanted counts (tile histogram) and their prefix sum.
// Spare room: half the tile's own count, 64, and a quarter of what its six
// face neighbours hold (particles diffuse in across steep density edges).
// The overflow bin keeps capacity ovf_cap.  One block.
__device__ __forceinline__ void layout_body(const int* __restrict__ want, int* __restrict__ cap,
                                            long long* __restrict__ base, int NT, int ntx, int ovf_cap) {
  __shared__ long long s_part[1024];
  const int per = (NT + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  long long local = 0;
  for (int b = b0; b < min(b0 + per, NT); ++b) {
    const int w = want[b];
    const int tz = b % ntx, ty = (b / ntx) % ntx, tx = b / (ntx * ntx);
    long long nsum = 0;
    for (int d = -1; d <= 1; d += 2) {
      nsum += want[((((tx + d + ntx) % ntx) * ntx) + ty) * ntx + tz];
      nsum += want[((tx * ntx) + (ty + d + ntx) % ntx) * ntx + tz];
      nsum += want[((tx * ntx) + ty) * ntx + (tz + d + ntx) % ntx];
    }
    long long cl = (long long)w + w / 2 + 64 + nsum / 4;
    cl = cl < 0x7ffffff0LL ? cl : 0x7ffffff0LL;
    const int c = (int)((cl + 3) & ~3LL);   // 4-slot multiples keep every bin 16-byte aligned
    cap[b] = c;
    local += c;
  }
  s_part[threadIdx.x] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    const long long v = threadIdx.x >= (unsigned)off ? s_part[threadIdx.x - off] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = s_part[threadIdx.x] - local;
  for (int b = b0; b < min(b0 + per, NT); ++b) {
    base[b] = run;
    run += cap[b];
  }
  if (threadIdx.x == blockDim.x - 1) {
    base[NT] = s_part[threadIdx.x];
    cap[NT] = (ovf_cap + 3) & ~3;
  }
}

__global__ void __launch_bounds__(1024)
k_layout(const int* __restrict__ want, int* __restrict__ cap, long long* __restrict__ base, int NT, int ntx,
         int ovf_cap) {
  layout_body(want, cap, base, NT, ntx, ovf_cap);
}

// One block per run.
__global__ void __launch_bounds__(1024) k_layout_batch(const LayoutArgs* __restrict__ t) {
  const LayoutArgs& a = t[blockIdx.x];
  layout_body(a.want, a.cap, a.base, a.NT, a.ntx, a.ovf_cap);
}

// Tile histogram of plain (unbinned) positions.  With few enough tiles each
// block counts its contiguous range in shared memory and adds its counts to
// the global histogram once; otherwise warps aggregate equal tiles.
template <typename T>
__global__ void __launch_bounds__(256)
k_tile_hist(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, Geo<T> g,
            int shift, int ntx, int NT, int* __restrict__ hist, int use_smem) {
  extern __shared__ int s_cnt[];
  const int lane = threadIdx.x & 31;
  if (use_smem) {
    for (int t = threadIdx.x; t < NT; t += blockDim.x) s_cnt[t] = 0;
    __syncthreads();
    const int64_t per = (P + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(P, b0 + per);
    for (int64_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) {
      int cx, cy, cz;
      T l;
      cell_lambda(x[p], g, cx, l);
      cell_lambda(y[p], g, cy, l);
      cell_lambda(z[p], g, cz, l);
      atomicAdd(s_cnt + tile_of(cx & g.mask, cy & g.mask, cz & g.mask, shift, ntx), 1);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NT; t += blockDim.x)
      if (s_cnt[t]) atomicAdd(hist + t, s_cnt[t]);
    return;
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_iter = (P + stride - 1) / stride;
  for (int64_t it = 0; it < n_iter; ++it) {
    const int64_t p = it * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < P;
    unsigned key = 0xFFFFFFFFu;
    if (valid) {
      int cx, cy, cz;
      T l;
      cell_lambda(x[p], g, cx, l);
      cell_lambda(y[p], g, cy, l);
      cell_lambda(z[p], g, cz, l);
      key = (unsigned)tile_of(cx & g.mask, cy & g.mask, cz & g.mask, shift, ntx);
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, key);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(hist + key, __popc(peers));
  }
}

// Re-bin plain (particle-order) arrays into tile bins.  Each block takes a
// contiguous range, counts its tiles in shared memory, reserves one range per
// tile in the destination bins with a single global atomic, and hands out the
// slots of that range with shared atomics.  Must run with the same grid as
// nothing else depends on the order inside a bin.
template <typename T>
__global__ void __launch_bounds__(256)
k_rebin_plain(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z,
              const uint32_t* __restrict__ id, int64_t P, Geo<T> g, int shift, int ntx, int NT,
              T* __restrict__ dx, T* __restrict__ dy, T* __restrict__ dz, uint32_t* __restrict__ did,
              const long long* __restrict__ dst_base, const int* __restrict__ dst_cap, int* __restrict__ dst_cursor,
              int* err, int64_t id0, int wrap) {
  extern __shared__ int s_cnt[];
  for (int t = threadIdx.x; t < NT; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();
  const int64_t per = (P + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(P, b0 + per);
  // positions, wrapped into the box if asked (the periodic wrap of uploaded data)
  auto pos = [&](const T* a, int64_t p) { return wrap ? wrap_coord(a[p], g) : a[p]; };
  auto tile = [&](int64_t p) {
    int cx, cy, cz;
    T l;
    cell_lambda(pos(x, p), g, cx, l);
    cell_lambda(pos(y, p), g, cy, l);
    cell_lambda(pos(z, p), g, cz, l);
    return tile_of(cx & g.mask, cy & g.mask, cz & g.mask, shift, ntx);
  };
  for (int64_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) atomicAdd(s_cnt + tile(p), 1);
  __syncthreads();
  for (int t = threadIdx.x; t < NT; t += blockDim.x)
    if (s_cnt[t]) s_cnt[t] = atomicAdd(dst_cursor + t, s_cnt[t]);
  __syncthreads();
  for (int64_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) {
    const int t = tile(p);
    const int r = atomicAdd(s_cnt + t, 1);
    long long slot;
    if (r < dst_cap[t]) {
      slot = dst_base[t] + r;
    } else {
      const int o = atomicAdd(dst_cursor + NT, 1);
      slot = o < dst_cap[NT] ? dst_base[NT] + o : -1;
    }
    if (slot >= 0) {
      dx[slot] = pos(x, p);
      dy[slot] = pos(y, p);
      dz[slot] = pos(z, p);
      did[slot] = id ? id[p] : (uint32_t)(id0 + p);
    } else {
      atomicOr(err, 2);
    }
  }
}

// Read-back through a slot map: slot_of[id] = slot of particle id in the
// current bins (one 4-byte store per particle, the map L2-resident), then
// out[id] = X[slot_of[id]] over ids in order, so the output (host memory the
// device can address) is written whole lines at a time.
template <typename T>
__global__ void __launch_bounds__(256) k_slot_map(BinArgs<T> a, uint32_t* __restrict__ slot_of) {
  const long long c = blockIdx.x;
  if (c >= a.chunk_start[a.NT + 1]) return;
  const ChunkDesc d = a.chunks[c];
  item_slots(a, d, [&](long long s) { slot_of[a.sid[s]] = (uint32_t)s; });
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gather_slots(const uint32_t* __restrict__ slot_of, const T* __restrict__ bx, const T* __restrict__ by,
               const T* __restrict__ bz, int64_t P, T* __restrict__ ox, T* __restrict__ oy, T* __restrict__ oz) {
  // four ids per thread and iteration, their gathers issued together
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P; i0 += U * stride) {
    uint32_t s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s[u] = i0 + u * stride < P ? slot_of[i0 + u * stride] : 0u;
    T vx[U], vy[U], vz[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * stride < P) {
        vx[u] = bx[s[u]];
        vy[u] = by[s[u]];
        vz[u] = bz[s[u]];
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (i0 + u * stride < P) {
        ox[i0 + u * stride] = vx[u];
        oy[i0 + u * stride] = vy[u];
        oz[i0 + u * stride] = vz[u];
      }
  }
}

// The current bins' particles copied into contiguous arrays (x, y, z, id),
// each work item's particles kept together in bin order, so consecutive
// entries lie in the same grid tile; items land in the order their blocks
// reserve their ranges (cursor: zeroed before the launch).
template <typename T>
__global__ void __launch_bounds__(1024)
k_compact(BinArgs<T> a, unsigned long long* cursor, T* __restrict__ ox, T* __restrict__ oy, T* __restrict__ oz,
          uint32_t* __restrict__ oid) {
  __shared__ long long s_base;
  const long long c = blockIdx.x;
  if (c >= a.chunk_start[a.NT + 1]) return;
  const ChunkDesc d = a.chunks[c];
  if (threadIdx.x == 0) s_base = (long long)atomicAdd(cursor, (unsigned long long)d.len);
  __syncthreads();
  long long o = s_base;
  auto copy_run = [&](long long s0, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      ox[o + i] = a.sx[s0 + i];
      oy[o + i] = a.sy[s0 + i];
      oz[o + i] = a.sz[s0 + i];
      oid[o + i] = a.sid[s0 + i];
    }
    o += n;
  };
  if (d.bin >= 0) {
    copy_run(d.start, d.len);
    return;
  }
  const int m = merge_of(d);
  for (int k = 0; k < m; ++k) {
    const int b = (int)d.start * m + k;
    if (b > a.NT) break;
    const int n = a.src_count[b];
    if (bin_is_small(b, n, a.NT)) copy_run(a.src_base[b], n);
  }
}

// Scatter binned particles back to particle order: out[id] = X[slot].
template <typename T>
__global__ void __launch_bounds__(256)
k_unbin(BinArgs<T> a, T* __restrict__ ox, T* __restrict__ oy, T* __restrict__ oz) {
  const long long c = blockIdx.x;
  if (c >= a.chunk_start[a.NT + 1]) return;
  const ChunkDesc d = a.chunks[c];
  item_slots(a, d, [&](long long s) {
    const uint32_t id = a.sid[s];
    ox[id] = a.sx[s];
    oy[id] = a.sy[s];
    oz[id] = a.sz[s];
  });
}

// Gather back to particle order in two coalesced-friendly passes: each
// particle's (x, y, z) goes to its id's slot of a 4-wide scratch array (one
// 16- or 32-byte store instead of three scattered 4- or 8-byte ones), then
// the scratch is transposed into the three output arrays.
template <typename T> struct Vec4Store;
template <> struct Vec4Store<float> {
  static __device__ __forceinline__ void put(float* dst, float x, float y, float z) {
    *reinterpret_cast<float4*>(dst) = make_float4(x, y, z, 0.f);
  }
};
template <> struct Vec4Store<double> {
  static __device__ __forceinline__ void put(double* dst, double x, double y, double z) {
    reinterpret_cast<double2*>(dst)[0] = make_double2(x, y);
    reinterpret_cast<double2*>(dst)[1] = make_double2(z, 0.0);
  }
};

template <typename T>
__global__ void __launch_bounds__(256) k_unbin_aos(BinArgs<T> a, T* __restrict__ aos) {
  const long long c = blockIdx.x;
  if (c >= a.chunk_start[a.NT + 1]) return;
  const ChunkDesc d = a.chunks[c];
  item_slots(a, d, [&](long long s) { Vec4Store<T>::put(aos + (size_t)a.sid[s] * 4, a.sx[s], a.sy[s], a.sz[s]); });
}

// Read-back in particle order, step 1: the particles of the current bins
// partitioned by id into the host copy's pieces (piece k: ids
// [pb.b[k], pb.b[k+1])) as SoA records, piece k's at pb.b[k] on.  A block
// takes one work item, counts its particles per piece in shared memory,
// reserves each piece's range with one global atomic and writes.  The ids
// are a permutation of 0 .. P-1, so piece k receives exactly its own range.
template <typename T>
__global__ void __launch_bounds__(256)
k_partition_pieces(BinArgs<T> a, PieceBounds pb, int* __restrict__ cursor, T* __restrict__ rx, T* __restrict__ ry,
                   T* __restrict__ rz, uint32_t* __restrict__ rid) {
  __shared__ int cnt[PieceBounds::kMax], base[PieceBounds::kMax];
  const long long c = blockIdx.x;
  if (c >= a.chunk_start[a.NT + 1]) return;
  const ChunkDesc d = a.chunks[c];
  auto piece_of = [&](uint32_t id) {
    int k = pb.np - 1;
    while (k > 0 && (long long)id < pb.b[k]) --k;
    return k;
  };
  if (threadIdx.x < PieceBounds::kMax) cnt[threadIdx.x] = 0;
  __syncthreads();
  item_slots(a, d, [&](long long s) { atomicAdd(&cnt[piece_of(a.sid[s])], 1); });
  __syncthreads();
  if (threadIdx.x < pb.np) {
    const int n = cnt[threadIdx.x];
    base[threadIdx.x] = n ? atomicAdd(cursor + threadIdx.x, n) : 0;
    cnt[threadIdx.x] = 0;
  }
  __syncthreads();
  item_slots(a, d, [&](long long s) {
    const uint32_t id = a.sid[s];
    const int k = piece_of(id);
    const long long o = pb.b[k] + base[k] + atomicAdd(&cnt[k], 1);
    rx[o] = a.sx[s];
    ry[o] = a.sy[s];
    rz[o] = a.sz[s];
    rid[o] = id;
  });
}

// Step 2, per piece: its records scattered to their particles' slots.  A
// piece's slots span 1/8 of the output arrays, small enough to stay in L2
// while its partial sectors fill.
template <typename T>
__global__ void __launch_bounds__(256)
k_scatter_piece(const T* __restrict__ rx, const T* __restrict__ ry, const T* __restrict__ rz,
                const uint32_t* __restrict__ rid, int64_t a0, int64_t n, int64_t P, T* __restrict__ ox,
                T* __restrict__ oy, T* __restrict__ oz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = a0 + i;
    const uint32_t id = rid[s];
    if ((int64_t)id < P) {
      ox[id] = rx[s];
      oy[id] = ry[s];
      oz[id] = rz[s];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_aos4_to_soa(const T* __restrict__ aos, int64_t P, T* __restrict__ ox, T* __restrict__ oy, T* __restrict__ oz) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    const T* v = aos + (size_t)p * 4;
    ox[p] = v[0];
    oy[p] = v[1];
    oz[p] = v[2];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_iota(uint32_t* id, int64_t P) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) id[p] = (uint32_t)p;
}

// ---------------------------------------------------------------------------
// Stand-alone operators (stateless entry points).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_deposit(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, Geo<T> g, T w,
          T* __restrict__ phi, int order) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    int cx, cy, cz;
    T lx, ly, lz;
    cell_lambda(x[p], g, cx, lx);
    cell_lambda(y[p], g, cy, ly);
    cell_lambda(z[p], g, cz, lz);
    stencil_visit_global<T>(order, cx, cy, cz, lx, ly, lz, w, g, [&](int idx, T f) { atomicAdd(phi + idx, f); });
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_gather(const T* __restrict__ x, const T* __restrict__ y, const T* __restrict__ z, int64_t P, Geo<T> g,
         const T* __restrict__ f, int ncomp, int order, T* __restrict__ out) {
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
      stencil_visit_global<T>(order, cx, cy, cz, lx, ly, lz, T(1), g,
                              [&](int idx, T wt) { acc += wt * f[c * N + idx]; });
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

template <typename T>
__global__ void __launch_bounds__(256) k_wrap_soa(int64_t P, Geo<T> g, T* x, T* y, T* z) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    x[p] = wrap_coord(x[p], g);
    y[p] = wrap_coord(y[p], g);
    z[p] = wrap_coord(z[p], g);
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
    const cpx<T> v = alpha[i];
    const double e = mult * ((double)v.x * v.x + (double)v.y * v.y);
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
// Launchers.
// ---------------------------------------------------------------------------
int binned_window_slots(int H) { return H <= 16 ? kReplicas * H * H * H : kTileReps * kWinSlots; }
int binned_chunk() { return kChunk; }
int binned_tile_shift(int H) { return H <= 16 ? 30 : kTileShift; }

template <typename T, bool FIXED, bool MOVE, bool DEPOSIT, bool REBIN>
static cudaError_t launch_binned_t(const BinArgs<T>& a, cudaStream_t s) {
  const bool whole = a.g.H <= 16;
  const size_t smem = DEPOSIT ? (size_t)binned_window_slots(a.g.H) * sizeof(typename WinType<T>::type) : 0;
  auto kern = whole ? k_binned<T, FIXED, MOVE, DEPOSIT, REBIN, true> : k_binned<T, FIXED, MOVE, DEPOSIT, REBIN, false>;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem)) != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  kern<<<sms * per_sm, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_binned(const BinArgs<T>& a, int move, int deposit, int rebin, cudaStream_t s) {
  if (a.fixed) {
    if (move && !deposit && rebin) return launch_binned_t<T, true, true, false, true>(a, s);
    if (!move && deposit && !rebin) return launch_binned_t<T, true, false, true, false>(a, s);
    if (!move && !deposit && rebin) return launch_binned_t<T, true, false, false, true>(a, s);
  } else {
    if (move && !deposit && rebin) return launch_binned_t<T, false, true, false, true>(a, s);
    if (!move && deposit && !rebin) return launch_binned_t<T, false, false, true, false>(a, s);
    if (!move && !deposit && rebin) return launch_binned_t<T, false, false, false, true>(a, s);
  }
  return cudaErrorInvalidValue;
}

int chunk_list_blocks(int NT) { return (NT + 1 + kCLBlock - 1) / kCLBlock; }

cudaError_t launch_chunk_list(const ChunkListArgs& a, unsigned long long* work, unsigned long long* ovf_total,
                              cudaStream_t s) {
  const int nblk = chunk_list_blocks(a.NT);
  k_chunk_count<<<nblk, kCLBlock, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_chunk_emit<<<nblk, kCLBlock, 0, s>>>(a, work, ovf_total);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_move_batch(const BinArgs<T>* table, const long long* prefix, int nruns, unsigned long long* work,
                              const uint32_t* step, bool move, cudaStream_t s, int blocks_per_sm, int g2p) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  // the gather order fixed at compile time when every run uses the same one
  auto k = !move ? k_move_batch<T, false, 0>
                 : (g2p == 2 ? k_move_batch<T, true, 2> : g2p == 4 ? k_move_batch<T, true, 4> : k_move_batch<T, true, 0>);
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMoveThreads, 0)) != cudaSuccess) return e;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  k<<<sms * per_sm, kMoveThreads, 0, s>>>(table, prefix, nruns, work, step);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit_batch(const BinArgs<T>* table, const long long* prefix, int nruns,
                                 unsigned long long* work, bool fixed, cudaStream_t s, int blocks_per_sm) {
  const size_t smem = (size_t)kTileReps * kWinSlots * sizeof(typename WinType<T>::type);
  auto k = fixed ? k_deposit_batch<T, true> : k_deposit_batch<T, false>;
  cudaError_t e;
  if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem)) != cudaSuccess) return e;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  if (per_sm < 1) per_sm = 1;
  k<<<sms * per_sm, 256, smem, s>>>(table, prefix, nruns, work);
  return cudaGetLastError();
}

cudaError_t launch_chunk_list_batch(const ChunkListArgs* t, int nruns, int max_NT, cudaStream_t s) {
  const dim3 grid(chunk_list_blocks(max_NT), nruns);
  k_chunk_count_batch<<<grid, kCLBlock, 0, s>>>(t);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_chunk_emit_batch<<<grid, kCLBlock, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_run_prefix(const ChunkListArgs* t, int nruns, long long* prefix, unsigned long long* work,
                              uint32_t* step, int bump, cudaStream_t s) {
  k_run_prefix<<<1, 1024, 0, s>>>(t, nruns, prefix, work, step, bump);
  return cudaGetLastError();
}

cudaError_t launch_layout_batch(const LayoutArgs* t, int nruns, cudaStream_t s) {
  k_layout_batch<<<nruns, 1024, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_layout(const int* want, int* cap, long long* base, int NT, int ntx, int ovf_cap, cudaStream_t s) {
  k_layout<<<1, 1024, 0, s>>>(want, cap, base, NT, ntx, ovf_cap);
  return cudaGetLastError();
}

static int plain_blocks(int64_t P) {
  int b = grid_for(P, 2048);
  return b > 152 * 8 ? 152 * 8 : b;
}
static constexpr int kMaxSmemTiles = 8192;

template <typename T>
cudaError_t launch_tile_hist(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, int shift, int ntx, int NT,
                             int* hist, cudaStream_t s) {
  const int use_smem = NT <= kMaxSmemTiles ? 1 : 0;
  const int b = use_smem ? plain_blocks(P) : (grid_for(P, 256) > 152 * 16 ? 152 * 16 : grid_for(P, 256));
  k_tile_hist<T><<<b, 256, use_smem ? NT * sizeof(int) : 0, s>>>(x, y, z, P, g, shift, ntx, NT, hist, use_smem);
  return cudaGetLastError();
}

template <typename T>
bool launch_rebin_plain(const T* x, const T* y, const T* z, const uint32_t* id, int64_t P, Geo<T> g, int shift,
                        int ntx, int NT, T* dx, T* dy, T* dz, uint32_t* did, const long long* dst_base,
                        const int* dst_cap, int* dst_cursor, int* err, cudaStream_t s, cudaError_t* e, int64_t id0,
                        bool wrap) {
  if (NT > kMaxSmemTiles) return false;
  k_rebin_plain<T><<<plain_blocks(P), 256, NT * sizeof(int), s>>>(x, y, z, id, P, g, shift, ntx, NT, dx, dy, dz, did,
                                                                 dst_base, dst_cap, dst_cursor, err, id0,
                                                                 wrap ? 1 : 0);
  *e = cudaGetLastError();
  return true;
}

int rebin_plain_max_tiles() { return kMaxSmemTiles; }

template <typename T>
cudaError_t launch_unbin_aos(const BinArgs<T>& a, int64_t max_chunks, T* aos, cudaStream_t s) {
  k_unbin_aos<T><<<(unsigned)max_chunks, 256, 0, s>>>(a, aos);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_partition_pieces(const BinArgs<T>& a, int64_t max_chunks, const PieceBounds& pb, int* cursor, T* rx,
                                    T* ry, T* rz, uint32_t* rid, cudaStream_t s) {
  if (pb.np < 1 || pb.np > PieceBounds::kMax) return cudaErrorInvalidValue;
  if (max_chunks < 1) return cudaSuccess;
  k_partition_pieces<T><<<(unsigned)max_chunks, 256, 0, s>>>(a, pb, cursor, rx, ry, rz, rid);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_compact(const BinArgs<T>& a, int64_t max_chunks, unsigned long long* cursor, T* x, T* y, T* z,
                           uint32_t* id, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess || max_chunks < 1) return e;
  k_compact<T><<<(unsigned)max_chunks, 1024, 0, s>>>(a, cursor, x, y, z, id);   // a work item per block
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_read_back_mapped(const BinArgs<T>& a, int64_t max_chunks, uint32_t* slot_of, int64_t P, T* x, T* y,
                                   T* z, cudaStream_t s) {
  if (max_chunks < 1 || P < 1) return cudaSuccess;
  k_slot_map<T><<<(unsigned)max_chunks, 256, 0, s>>>(a, slot_of);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t b = (P + 255) / 256;
  k_gather_slots<T><<<(unsigned)(b > 152 * 16 ? 152 * 16 : b), 256, 0, s>>>(slot_of, a.sx, a.sy, a.sz, P, x, y, z);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_piece(const T* rx, const T* ry, const T* rz, const uint32_t* rid, int64_t a0, int64_t n,
                                 int64_t P, T* x, T* y, T* z, cudaStream_t s) {
  if (n < 1) return cudaSuccess;
  const int64_t b = (n + 255) / 256;
  k_scatter_piece<T><<<(unsigned)(b > 152 * 8 ? 152 * 8 : b), 256, 0, s>>>(rx, ry, rz, rid, a0, n, P, x, y, z);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_aos4_to_soa(const T* aos, int64_t P, T* x, T* y, T* z, cudaStream_t s) {
  const int64_t b = (P + 255) / 256;
  k_aos4_to_soa<T><<<(unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)), 256, 0, s>>>(aos, P, x, y, z);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unbin(const BinArgs<T>& a, int64_t max_chunks, T* x, T* y, T* z, T* aos_scratch, int64_t P,
                         cudaStream_t s) {
  if (!aos_scratch) {
    k_unbin<T><<<(unsigned)max_chunks, 256, 0, s>>>(a, x, y, z);
    return cudaGetLastError();
  }
  k_unbin_aos<T><<<(unsigned)max_chunks, 256, 0, s>>>(a, aos_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t b = (P + 255) / 256;
  k_aos4_to_soa<T><<<(unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b)), 256, 0, s>>>(aos_scratch, P, x, y, z);
  return cudaGetLastError();
}

cudaError_t launch_iota(uint32_t* id, int64_t P, cudaStream_t s) {
  k_iota<int><<<grid_for(P, 256), 256, 0, s>>>(id, P);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_deposit(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, T w, T* phi, int order,
                           cudaStream_t s) {
  k_deposit<T><<<grid_for(P, 256), 256, 0, s>>>(x, y, z, P, g, w, phi, order);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const T* x, const T* y, const T* z, int64_t P, Geo<T> g, const T* f, int ncomp, int order,
                          T* out, cudaStream_t s) {
  k_gather<T><<<grid_for(P, 256), 256, 0, s>>>(x, y, z, P, g, f, ncomp, order, out);
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

template <typename T> cudaError_t launch_wrap_soa(int64_t P, Geo<T> g, T* x, T* y, T* z, cudaStream_t s) {
  k_wrap_soa<T><<<grid_for(P, 256), 256, 0, s>>>(P, g, x, y, z);
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
  template cudaError_t launch_binned<T>(const BinArgs<T>&, int, int, int, cudaStream_t);                       \
  template cudaError_t launch_move<T>(const BinArgs<T>&, cudaStream_t);                                       \
  template cudaError_t launch_move_batch<T>(const BinArgs<T>*, const long long*, int, unsigned long long*,     \
                                            const uint32_t*, bool, cudaStream_t, int, int);                  \
  template cudaError_t launch_deposit_batch<T>(const BinArgs<T>*, const long long*, int, unsigned long long*,  \
                                               bool, cudaStream_t, int);                                      \
  template cudaError_t launch_tile_hist<T>(const T*, const T*, const T*, int64_t, Geo<T>, int, int, int, int*, \
                                           cudaStream_t);                                                    \
  template bool launch_rebin_plain<T>(const T*, const T*, const T*, const uint32_t*, int64_t, Geo<T>, int, int, \
                                      int, T*, T*, T*, uint32_t*, const long long*, const int*, int*, int*,    \
                                      cudaStream_t, cudaError_t*, int64_t, bool);                             \
  template cudaError_t launch_unbin_aos<T>(const BinArgs<T>&, int64_t, T*, cudaStream_t);                     \
  template cudaError_t launch_aos4_to_soa<T>(const T*, int64_t, T*, T*, T*, cudaStream_t);                    \
  template cudaError_t launch_partition_pieces<T>(const BinArgs<T>&, int64_t, const PieceBounds&, int*, T*, T*, \
                                                  T*, uint32_t*, cudaStream_t);                                \
  template cudaError_t launch_scatter_piece<T>(const T*, const T*, const T*, const uint32_t*, int64_t, int64_t, \
                                               int64_t, T*, T*, T*, cudaStream_t);                             \
  template cudaError_t launch_read_back_mapped<T>(const BinArgs<T>&, int64_t, uint32_t*, int64_t, T*, T*, T*, \
                                                  cudaStream_t);                                              \
  template cudaError_t launch_compact<T>(const BinArgs<T>&, int64_t, unsigned long long*, T*, T*, T*, uint32_t*, \
                                         cudaStream_t);                                                       \
  template cudaError_t launch_unbin<T>(const BinArgs<T>&, int64_t, T*, T*, T*, T*, int64_t, cudaStream_t);    \
  template cudaError_t launch_deposit<T>(const T*, const T*, const T*, int64_t, Geo<T>, T, T*, int,           \
                                         cudaStream_t);                                                      \
  template cudaError_t launch_gather<T>(const T*, const T*, const T*, int64_t, Geo<T>, const T*, int, int,   \
                                        T*, cudaStream_t);                                                   \
  template cudaError_t launch_noise<T>(uint64_t, int64_t, int64_t, int64_t, T*, cudaStream_t);               \
  template cudaError_t launch_moments<T>(const T*, const T*, const T*, int64_t, double*, cudaStream_t);      \
  template cudaError_t launch_aos_to_soa<T>(const double*, int64_t, Geo<T>, T*, T*, T*, cudaStream_t);       \
  template cudaError_t launch_wrap_soa<T>(int64_t, Geo<T>, T*, T*, T*, cudaStream_t);                        \
  template cudaError_t launch_alpha_energy<T>(const cpx<T>*, int, double*, cudaStream_t);
SIPF_INST(float)
SIPF_INST(double)
#undef SIPF_INST

}  // namespace sipf
