// C ABI of libsipf: parameter validation, the context (device state of one
// SIPF-PIC run), the step loop of Algorithm 4 and the stateless operators.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sipf.h"
#include "sipf_internal.h"

using namespace sipf;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? SIPF_ENOMEM : SIPF_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define SIPF_CK(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// H0 = ceil(8 H^(8/13) L^(5/13)) (Sec. 5.1).  With H = 2^h and L = a 2^e (a
// odd), x^13 = 2^(39 + 8h + 5e) a^5, so x is an integer exactly when a = c^13
// for an odd integer c (c <= 15 for a 53-bit a) and 13 divides t = 39 + 8h + 5e
// with t >= 0; then x = 2^(t/13) c^5.  That case is returned exactly (a
// floating-point power can land just above the integer, e.g. 64.00000000000001
// at H = L = 8, and its ceiling would be one too large); otherwise x is not an
// integer and the ceiling of the floating-point value is taken.
double auto_H0(int H, double L) {
  const double x = 8.0 * pow((double)H, 8.0 / 13.0) * pow(L, 5.0 / 13.0);
  int e = 0;
  const double fr = frexp(L, &e);
  uint64_t a = (uint64_t)ldexp(fr, 53);
  int e2 = e - 53;
  while (a && !(a & 1)) {
    a >>= 1;
    ++e2;
  }
  int h = 0;
  while ((1 << h) < H) ++h;
  const long t = 39L + 8L * h + 5L * e2;
  if (t >= 0 && t % 13 == 0) {
    for (uint64_t c = 1; c <= 15; c += 2) {
      uint64_t c13 = 1;
      for (int i = 0; i < 13; ++i) c13 *= c;
      if (c13 == a) return ldexp((double)(c * c * c * c * c), (int)(t / 13));
    }
  }
  return ceil(x);
}

double effective_H0(const sipf_params& p) {
  if (p.H0 < 0) return auto_H0(p.H, p.L);
  return p.H0;
}

int validate(const sipf_params* p) {
  if (!p) return fail(SIPF_EINVAL, "params is NULL");
  auto bad = [](const char* f) { return fail(SIPF_EINVAL, std::string("invalid parameter: ") + f); };
  if (!(p->P >= 1 && p->P <= (1LL << 30))) return bad("P (1 <= P <= 2^30)");
  if (!is_pow2(p->H) || p->H < 8 || p->H > kNmax) return bad("H (power of two in [8, 256])");
  if (p->precision != 32 && p->precision != 64) return bad("precision (32 or 64)");
  if (!(isfinite(p->L) && p->L > 0)) return bad("L (> 0)");
  if (!(isfinite(p->dt) && p->dt > 0)) return bad("dt (> 0)");
  if (!(isfinite(p->eps) && p->eps > 0)) return bad("eps (> 0)");
  if (!(isfinite(p->mu) && p->mu >= 0)) return bad("mu (>= 0)");
  if (!(isfinite(p->chi) && p->chi >= 0)) return bad("chi (>= 0)");
  if (!(isfinite(p->k) && p->k >= 0)) return bad("k (>= 0)");
  if (!(isfinite(p->mass) && p->mass > 0)) return bad("mass (> 0)");
  if (!(isfinite(p->T) && p->T >= 0)) return bad("T (>= 0)");
  if (!isfinite(p->H0)) return bad("H0 (finite)");
  if (p->p2g_order != 2 && p->p2g_order != 4) return bad("p2g_order (2 or 4)");
  if (p->g2p_order != 2 && p->g2p_order != 4) return bad("g2p_order (2 or 4)");
  if (p->splitting != SIPF_SPLIT_HALF && p->splitting != SIPF_SPLIT_PLAIN) return bad("splitting");
  if (p->deposit_mode != SIPF_DEPOSIT_ATOMIC && p->deposit_mode != SIPF_DEPOSIT_DETERMINISTIC)
    return bad("deposit_mode");
  if (p->propagator != SIPF_PROP_IMPLICIT && p->propagator != SIPF_PROP_EXP) return bad("propagator");
  if (p->resort_every < 0) return bad("resort_every (>= 0)");
  if (p->k == 0 && p->propagator == SIPF_PROP_IMPLICIT && p->eps / p->dt == 0) return bad("eps/dt");
  return SIPF_OK;
}

// Deterministic deposit: weights are summed as integers in units of 2^-K.
// float runs: K = 18 (an int32 shared window of 4096 particles cannot
// overflow); double runs: K = 61 - ceil(log2 P), capped at 40, so that even a
// node that gathered every particle stays inside int64.
// Fixed-point unit 2^-K of a stencil weight in the deterministic mode.  FP32:
// int32 shared windows whose copies receive at most 1024 particles of a
// 4096-particle work item (tile windows 896, whole-grid windows 1024), so
// 1024 * 2^19 < 2^30.  FP64: int64 throughout, the total of P particles.
int fixed_k(const sipf_params& p) {
  if (p.precision == 32) return 19;
  int lg = 0;
  while ((1LL << lg) < p.P + 1) ++lg;
  int k = 61 - lg;
  return k > 40 ? 40 : k;
}

}  // namespace

// Shared with the other translation units of the library (sipf_internal.h).
namespace sipf {
int report_error(int code, const std::string& msg) { return fail(code, msg); }
int report_cuda(cudaError_t e, const char* where) { return cuda_fail(e, where); }
double filter_scale(const sipf_params& p) { return effective_H0(p); }
}  // namespace sipf


struct sipf_ctx {
  sipf_params p{};
  double H0 = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0;
  size_t esz = 4;
  // particles: two tile-binned buffers (x, y, z, id) sharing one of two layouts
  int NT = 1, ntx = 1, shift = 30;
  int64_t cap_total = 0;
  void* bx[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  uint32_t* bid[2] = {nullptr, nullptr};
  int* lcap[2] = {nullptr, nullptr};
  long long* lbase[2] = {nullptr, nullptr};
  int* cursor[2] = {nullptr, nullptr};
  int* count = nullptr;
  long long* chunk_start = nullptr;
  ChunkDesc* chunks = nullptr;
  long long* part = nullptr;    // per-block chunk totals of the chunk-list passes
  unsigned long long* work = nullptr;
  unsigned long long* ovf = nullptr;   // particles found in the overflow bin while timing
  int* hist = nullptr;
  int cur = 0, lc = 0;            // current buffer, active layout
  int64_t since_layout = 0;
  // staging in particle order (x, y, z, id) and its one-bin description
  void* st[3] = {nullptr, nullptr, nullptr};
  uint32_t* st_id = nullptr;
  int* st_count = nullptr;
  int* st_cap = nullptr;
  long long* st_base = nullptr;
  // grid state
  void* phi = nullptr;     // H^3 T, or H^3 int64 (deterministic deposit)
  void* T1 = nullptr;      // S complex: forward intermediate
  void* alpha = nullptr;   // S complex: alpha^(n)
  void* T2 = nullptr;      // 3 S complex: gradient spectra
  void* grad = nullptr;    // 4 H^3 T: (gx, gy, gz, 0) per node; scratch between steps
  double* dsc = nullptr;   // FP64 accumulators (see kDsc*)
  int* err = nullptr;
  void* fft_run = nullptr; // device FftRun<T> of this context (H >= 32): the step's field solve
  // optional per-stage timing: 7 events per step (stage boundaries)
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  int64_t timed_steps = 0, timed_kernels = 0;
  int64_t launches = 0;
  // host-buffer transfers (sipf_upload_soa / sipf_download_soa) run in pieces
  // on two side streams so copies overlap the re-binning, the un-binning and
  // the step's last deposit; every transfer ends with the context stream
  // waiting for them
  cudaStream_t side[2] = {nullptr, nullptr};   // [0] kernels, [1] copies
  static constexpr int kPieces = PieceBounds::kMax;
  int* pcur = nullptr;     // per-piece cursors of the read-back partition
  cudaEvent_t ev_piece[kPieces] = {};
  cudaEvent_t ev_pos = nullptr;     // recorded once the current bins are final (before the deposit)
  cudaEvent_t ev_begin = nullptr, ev_done = nullptr;
  bool pos_ready = false;           // ev_pos describes the current bins
  // phi does not hold the deposit of the current positions yet: the deposit
  // is made when phi is next read (the next step's field solve, a density
  // query), so positions replaced before that (a host upload every step)
  // are not deposited twice; phi_zero: phi is known to be all zero
  bool dep_pending = false;
  bool phi_zero = false;
  int64_t H3() const { return (int64_t)p.H * p.H * p.H; }
  int64_t S() const { return (int64_t)p.H * p.H * (p.H / 2 + 1); }
  bool fixed() const { return p.deposit_mode == SIPF_DEPOSIT_DETERMINISTIC; }
  int64_t max_chunks() const { return p.P / binned_chunk() + NT + 2; }
  int resort() const { return p.resort_every > 0 ? p.resort_every : 16; }
  // bins per merge window of the chunk lists (small bins of a window form one
  // work item): 4 for a single run, 16 for the runs of a batch
  int merge = 4;
};

enum { kDscMass = 0, kDscAlpha0 = 1, kDscM2 = 2, kDscRing = 3, kDscHF = 4, kDscTot = 5, kDscMax = 6, kDscCount = 8 };

namespace {

SpecParams spec_params(const sipf_ctx* c) {
  SpecParams sp;
  sp.L = c->p.L;
  sp.inv_L3 = 1.0 / (c->p.L * c->p.L * c->p.L);
  sp.tau = c->p.dt;
  sp.eps = c->p.eps;
  sp.k2 = c->p.k * c->p.k;
  sp.H0 = c->H0;
  sp.beta0 = c->p.mass * sp.inv_L3;
  sp.propagator = c->p.propagator;
  return sp;
}

// deterministic grid: integer counts of 2^-K weight units, times M0/P
double fixed_in_scale(const sipf_ctx* c) { return c->p.mass / (double)c->p.P * ldexp(1.0, -fixed_k(c->p)); }

// Arrays and parameters of the field solve of one run (batched FFT kernels).
template <typename T> FftRun<T> make_fft_run(const sipf_ctx* c) {
  FftRun<T> f;
  f.phi = c->phi;
  f.phi_fixed = c->fixed() ? 1 : 0;
  f.in_scale = fixed_in_scale(c);
  f.T1 = (cpx<T>*)c->T1;
  f.alpha = (cpx<T>*)c->alpha;
  f.T2 = (cpx<T>*)c->T2;
  f.grad = (T*)c->grad;
  f.sp = spec_params(c);
  f.shadow = c->dsc + kDscAlpha0;
  return f;
}

// Kernel arguments for src -> dst; src_buf < 0 selects the particle-order staging.
template <typename T> BinArgs<T> bin_args(sipf_ctx* c, int src_buf, int src_lay, int dst_buf, int dst_lay) {
  BinArgs<T> a{};
  if (src_buf < 0) {
    a.sx = (const T*)c->st[0];
    a.sy = (const T*)c->st[1];
    a.sz = (const T*)c->st[2];
    a.sid = c->st_id;
    a.src_base = c->st_base;
    a.src_count = c->st_count;
  } else {
    a.sx = (const T*)c->bx[src_buf][0];
    a.sy = (const T*)c->bx[src_buf][1];
    a.sz = (const T*)c->bx[src_buf][2];
    a.sid = c->bid[src_buf];
    a.src_base = c->lbase[src_lay];
    a.src_count = c->count;
  }
  a.chunk_start = c->chunk_start;
  a.chunks = c->chunks;
  if (dst_buf >= 0) {
    a.dx = (T*)c->bx[dst_buf][0];
    a.dy = (T*)c->bx[dst_buf][1];
    a.dz = (T*)c->bx[dst_buf][2];
    a.did = c->bid[dst_buf];
    a.dst_base = c->lbase[dst_lay];
    a.dst_cap = c->lcap[dst_lay];
    a.dst_cursor = c->cursor[dst_buf];
  }
  a.work = c->work;
  a.NT = c->NT;
  a.ntx = c->ntx;
  a.tile_shift = c->shift;
  a.phi = c->phi;
  a.grad4 = (const T*)c->grad;
  a.g = make_geo<T>(c->p.L, c->p.H);
  a.s_noise = (T)(c->p.splitting == SIPF_SPLIT_HALF ? sqrt(c->p.mu * c->p.dt) : sqrt(2.0 * c->p.mu * c->p.dt));
  a.chitau = (T)(c->p.chi * c->p.dt);
  a.wmass = (T)(c->p.mass / (double)c->p.P);
  a.fix_k = fixed_k(c->p);
  a.seed = c->p.seed;
  a.n = (uint32_t)(c->n + 1);
  a.p2g = c->p.p2g_order;
  a.g2p = c->p.g2p_order;
  a.split = c->p.splitting;
  a.fixed = c->fixed() ? 1 : 0;
  a.err = c->err;
  return a;
}

// Chunk-list arguments: bins of (cursor, cap, base) into the context's chunk
// arrays; `other` are the cursors to clear for the next pass.
ChunkListArgs cl_args(sipf_ctx* c, const int* cursor, const int* cap, const long long* base, int* other) {
  return ChunkListArgs{cursor, cap, base, c->count, c->chunk_start, c->chunks, other, c->NT, c->part, c->merge};
}

// The current bins are final (positions of step n, before their deposit):
// a download may start from here on a side stream.
cudaError_t mark_positions(sipf_ctx* c) {
  const cudaError_t e = cudaEventRecord(c->ev_pos, c->stream);
  c->pos_ready = e == cudaSuccess;
  return e;
}

// Pieces [a, b) of P particles for the pipelined host transfers.
inline int64_t piece_begin(int64_t P, int npieces, int k) { return P * k / npieces; }
inline int pieces_for(int64_t P) { return P >= (1 << 20) ? sipf_ctx::kPieces : 1; }

// The deposit of the current positions, if it is still owed (see
// dep_pending).  The work counter it uses was cleared by the chunk-list
// emission that made the current bins.
template <typename T> int flush_deposit(sipf_ctx* c) {
  if (!c->dep_pending) return SIPF_OK;
  if (!c->phi_zero)
    SIPF_CK(cudaMemsetAsync(c->phi, 0, (size_t)c->H3() * (c->fixed() ? 8 : sizeof(T)), c->stream));
  SIPF_CK(launch_binned<T>(bin_args<T>(c, c->cur, c->lc, -1, 0), 0, 1, 0, c->stream));
  c->launches += 1;
  c->dep_pending = false;
  c->phi_zero = false;
  return SIPF_OK;
}

// Bin the particle-order staging (wrapped positions and ids) into a fresh
// layout sized from its tile histogram; the deposit is owed.
template <typename T> int rebin_from_staging(sipf_ctx* c) {
  const int d = c->cur, L = 1 - c->lc;
  const size_t nb = (size_t)(c->NT + 1);
  SIPF_CK(cudaMemsetAsync(c->hist, 0, nb * sizeof(int), c->stream));
  SIPF_CK(launch_tile_hist<T>((const T*)c->st[0], (const T*)c->st[1], (const T*)c->st[2], c->p.P,
                              make_geo<T>(c->p.L, c->p.H), c->shift, c->ntx, c->NT, c->hist, c->stream));
  SIPF_CK(launch_layout(c->hist, c->lcap[L], c->lbase[L], c->NT, c->ntx, (int)c->p.P, c->stream));
  // chunk list of the staging (one bin holding all P particles); clears the destination cursors
  SIPF_CK(launch_chunk_list(cl_args(c, c->st_count, c->st_cap, c->st_base, c->cursor[d]), c->work, nullptr,
                            c->stream));
  cudaError_t e = cudaSuccess;
  if (!launch_rebin_plain<T>((const T*)c->st[0], (const T*)c->st[1], (const T*)c->st[2], c->st_id, c->p.P,
                             make_geo<T>(c->p.L, c->p.H), c->shift, c->ntx, c->NT, (T*)c->bx[d][0], (T*)c->bx[d][1],
                             (T*)c->bx[d][2], c->bid[d], c->lbase[L], c->lcap[L], c->cursor[d], c->err, c->stream,
                             &e)) {
    SIPF_CK(cudaMemsetAsync(c->work, 0, sizeof(unsigned long long), c->stream));
    e = launch_binned<T>(bin_args<T>(c, -1, 0, d, L), 0, 0, 1, c->stream);
  }
  SIPF_CK(e);
  SIPF_CK(launch_chunk_list(cl_args(c, c->cursor[d], c->lcap[L], c->lbase[L], c->cursor[1 - d]), c->work, nullptr,
                            c->stream));
  c->cur = d;
  c->lc = L;
  c->since_layout = 0;
  SIPF_CK(mark_positions(c));
  c->dep_pending = true;
  return SIPF_OK;
}

// Particle order -> staging arrays (or caller-owned device arrays).
template <typename T> int unbin_to(sipf_ctx* c, T* x, T* y, T* z) {
  // the other bin buffer is free between steps (the next move overwrites it):
  // its x array (cap_total >= 4P elements) is the 4-wide scratch
  SIPF_CK(launch_unbin<T>(bin_args<T>(c, c->cur, c->lc, -1, 0), c->max_chunks(), x, y, z,
                          (T*)c->bx[1 - c->cur][0], c->p.P, c->stream));
  return SIPF_OK;
}

template <typename T> int step_impl(sipf_ctx* c, int64_t nsteps) {
  const int H = c->p.H;
  const int nh = H / 2 + 1;
  const size_t S = (size_t)c->S();
  const SpecParams sp = spec_params(c);
  cpx<T>* T1 = (cpx<T>*)c->T1;
  cpx<T>* T2 = (cpx<T>*)c->T2;
  cpx<T>* al = (cpx<T>*)c->alpha;
  auto mark = [&](cudaEvent_t* slot) -> cudaError_t {
    if (!c->timing) return cudaSuccess;
    cudaError_t e = cudaEventCreate(slot);
    if (e == cudaSuccess) e = cudaEventRecord(*slot, c->stream);
    return e;
  };
  for (int64_t s = 0; s < nsteps; ++s) {
    cudaEvent_t ev[7] = {};
    const int64_t l0 = c->launches;
    SIPF_CK(mark(&ev[0]));
    // deposit X^(n-1) from its bins (Algorithm 2), owed since the last move or
    // upload
    { const int r = flush_deposit<T>(c); if (r) return r; }
    SIPF_CK(mark(&ev[1]));
    const FftRun<T>* fr = (const FftRun<T>*)c->fft_run;
    int fk = 0;   // field-solve kernels launched this step
    // beta^(n-1) = F_H I(rho-hat^(n-1)); the deposit grid is cleared as it is read
    if (fr) {
      SIPF_CK(launch_field_batch<T>(fr, 1, H, kFieldForward, c->stream, FieldTune{}, &fk));
    } else {
      SIPF_CK(launch_rows_r2c<T>(c->phi, c->fixed() ? 1 : 0, fixed_in_scale(c), true, T1, H, H * H, nullptr,
                                 c->stream));
      SIPF_CK(launch_cols<T>(T1, H, H, nh, 1, 0, -1, 1.0, c->stream));
    }
    c->phi_zero = true;
    SIPF_CK(mark(&ev[2]));
    // alpha^n and G(alpha^(n-1)), x axis back-transformed
    if (fr) {
      SIPF_CK(launch_field_batch<T>(fr, 1, H, kFieldSpectral, c->stream, FieldTune{}, &fk));
    } else {
      SIPF_CK(launch_spectral_x<T>(T1, al, T2, H, sp, kModeStep, c->dsc + kDscAlpha0, c->stream));
    }
    SIPF_CK(mark(&ev[3]));
    if (fr) {
      SIPF_CK(launch_field_batch<T>(fr, 1, H, kFieldInverse, c->stream, FieldTune{}, &fk));
    } else {
      SIPF_CK(launch_cols<T>(T2, H, H, nh, 3, S, +1, 1.0, c->stream));
      SIPF_CK(launch_rows_c2r<T>(T2, 3, S, (T*)c->grad, H, H * H, nullptr, c->stream));
    }
    SIPF_CK(mark(&ev[4]));
    // X^(n-1) -> X^n, re-bin into the other buffer by the new tile
    const int src = c->cur, dst = 1 - c->cur;
    // the move's work counter was cleared by the last chunk-list emission
    BinArgs<T> ma = bin_args<T>(c, src, c->lc, dst, c->lc);
    ma.work = c->work + 1;
    SIPF_CK(launch_move<T>(ma, c->stream));
    SIPF_CK(mark(&ev[5]));
    SIPF_CK(launch_chunk_list(cl_args(c, c->cursor[dst], c->lcap[c->lc], c->lbase[c->lc], c->cursor[src]), c->work,
                              c->timing ? c->ovf : nullptr, c->stream));
    c->launches += (fr ? fk : 5) + 3;
    c->cur = dst;
    c->n += 1;
    if (++c->since_layout >= c->resort()) {
      // new capacities from the tile counts just made, and a re-bin into them
      const int L = 1 - c->lc, d2 = 1 - c->cur;
      SIPF_CK(launch_layout(c->cursor[c->cur], c->lcap[L], c->lbase[L], c->NT, c->ntx, (int)c->p.P, c->stream));
      SIPF_CK(cudaMemsetAsync(c->work, 0, sizeof(unsigned long long), c->stream));
      SIPF_CK(launch_binned<T>(bin_args<T>(c, c->cur, c->lc, d2, L), 0, 0, 1, c->stream));
      SIPF_CK(launch_chunk_list(cl_args(c, c->cursor[d2], c->lcap[L], c->lbase[L], c->cursor[c->cur]), c->work, nullptr,
                                c->stream));
      c->launches += 4;
      c->cur = d2;
      c->lc = L;
      c->since_layout = 0;
    }
    SIPF_CK(mark_positions(c));
    SIPF_CK(mark(&ev[6]));
    // the deposit of X^n is made when phi is next read (the next step, or a
    // density query); an upload of new positions before then replaces it
    c->dep_pending = true;
    if (c->timing) {
      c->ev.insert(c->ev.end(), ev, ev + 7);
      c->timed_steps += 1;
      c->timed_kernels += c->launches - l0;
    }
  }
  return SIPF_OK;
}

// rho_num (filtered) or the plain deposited density into the grad scratch
// buffer as an H^3 real grid; FP64 mass sum and max into dsc.
template <typename T> int density_impl(sipf_ctx* c, int filtered, T** out_grid) {
  { const int r = flush_deposit<T>(c); if (r) return r; }
  const int H = c->p.H, nh = H / 2 + 1;
  const size_t S = (size_t)c->S();
  cpx<T>* T1 = (cpx<T>*)c->T1;
  cpx<T>* T2 = (cpx<T>*)c->T2;
  SpecParams sp = spec_params(c);
  if (!filtered) sp.H0 = 0.0;
  SIPF_CK(launch_rows_r2c<T>(c->phi, c->fixed() ? 1 : 0, fixed_in_scale(c), false, T1, H, H * H,
                             c->dsc + kDscMass, c->stream));
  SIPF_CK(launch_cols<T>(T1, H, H, nh, 1, 0, -1, 1.0, c->stream));
  SIPF_CK(launch_spectral_x<T>(T1, (cpx<T>*)c->alpha, T2, H, sp, kModeDensity, nullptr, c->stream));
  SIPF_CK(launch_cols<T>(T2, H, H, nh, 1, S, +1, 1.0, c->stream));
  SIPF_CK(launch_rows_c2r<T>(T2, 1, S, (T*)c->grad, H, H * H, c->dsc + kDscMax, c->stream));
  *out_grid = (T*)c->grad;
  return SIPF_OK;
}

template <typename T> int copy_grid_to_host(sipf_ctx* c, const T* dev, int64_t count, double* out, double scale) {
  std::vector<T> h((size_t)count);
  SIPF_CK(cudaMemcpyAsync(h.data(), dev, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < count; ++i) out[i] = (double)h[(size_t)i] * scale;
  return SIPF_OK;
}

template <typename T> int density_host(sipf_ctx* c, double* out, int filtered) {
  { const int r = flush_deposit<T>(c); if (r) return r; }
  const double h3 = pow(c->p.L / c->p.H, 3);
  if (!filtered) {
    // I rho-hat / h^3 straight from the deposit grid
    if (c->fixed()) {
      std::vector<long long> h((size_t)c->H3());
      SIPF_CK(cudaMemcpyAsync(h.data(), c->phi, h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
      SIPF_CK(cudaStreamSynchronize(c->stream));
      const double sc = fixed_in_scale(c) / h3;
      for (size_t i = 0; i < h.size(); ++i) out[i] = (double)h[i] * sc;
      return SIPF_OK;
    }
    return copy_grid_to_host<T>(c, (const T*)c->phi, c->H3(), out, 1.0 / h3);
  }
  T* g = nullptr;
  int r = density_impl<T>(c, 1, &g);
  if (r) return r;
  return copy_grid_to_host<T>(c, g, c->H3(), out, 1.0);
}

template <typename T> int field_host(sipf_ctx* c, double* out) {
  const int H = c->p.H, nh = H / 2 + 1;
  const size_t S = (size_t)c->S();
  SpecParams sp = spec_params(c);
  SIPF_CK(launch_spectral_x<T>(nullptr, (cpx<T>*)c->alpha, (cpx<T>*)c->T2, H, sp, kModeField, nullptr, c->stream));
  SIPF_CK(launch_cols<T>((cpx<T>*)c->T2, H, H, nh, 1, S, +1, 1.0, c->stream));
  SIPF_CK(launch_rows_c2r<T>((cpx<T>*)c->T2, 1, S, (T*)c->grad, H, H * H, nullptr, c->stream));
  return copy_grid_to_host<T>(c, (const T*)c->grad, c->H3(), out, 1.0);
}

template <typename T> int gradient_host(sipf_ctx* c, double* out) {
  const int H = c->p.H, nh = H / 2 + 1;
  const size_t S = (size_t)c->S();
  SpecParams sp = spec_params(c);
  SIPF_CK(launch_spectral_x<T>(nullptr, (cpx<T>*)c->alpha, (cpx<T>*)c->T2, H, sp, kModeGradOnly, nullptr, c->stream));
  SIPF_CK(launch_cols<T>((cpx<T>*)c->T2, H, H, nh, 3, S, +1, 1.0, c->stream));
  SIPF_CK(launch_rows_c2r<T>((cpx<T>*)c->T2, 3, S, (T*)c->grad, H, H * H, nullptr, c->stream));
  const int64_t N = c->H3();
  std::vector<T> h((size_t)N * 4);
  SIPF_CK(cudaMemcpyAsync(h.data(), c->grad, h.size() * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  for (int d = 0; d < 3; ++d)
    for (int64_t i = 0; i < N; ++i) out[d * N + i] = (double)h[(size_t)i * 4 + d];
  return SIPF_OK;
}

template <typename T> int diagnostics_impl(sipf_ctx* c, sipf_diag* d) {
  const double neg_inf_key = -INFINITY;
  double init[kDscCount];
  SIPF_CK(cudaMemcpyAsync(init, c->dsc, sizeof(init), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  init[kDscMass] = 0;
  init[kDscM2] = init[kDscRing] = init[kDscHF] = init[kDscTot] = 0;
  {
    long long b;
    memcpy(&b, &neg_inf_key, 8);
    b ^= 0x7fffffffffffffffLL;   // order-preserving key of -inf
    memcpy(&init[kDscMax], &b, 8);
  }
  SIPF_CK(cudaMemcpyAsync(c->dsc, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
  T* g = nullptr;
  int r = density_impl<T>(c, c->H0 > 0 ? 1 : 0, &g);
  if (r) return r;
  r = unbin_to<T>(c, (T*)c->st[0], (T*)c->st[1], (T*)c->st[2]);
  if (r) return r;
  SIPF_CK(launch_moments<T>((T*)c->st[0], (T*)c->st[1], (T*)c->st[2], c->p.P, c->dsc + kDscM2, c->stream));
  SIPF_CK(launch_alpha_energy<T>((cpx<T>*)c->alpha, c->p.H, c->dsc + kDscHF, c->stream));
  double out[kDscCount];
  SIPF_CK(cudaMemcpyAsync(out, c->dsc, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  long long b;
  memcpy(&b, &out[kDscMax], 8);
  if (b < 0) b ^= 0x7fffffffffffffffLL;
  double mx;
  memcpy(&mx, &b, 8);
  d->mass = out[kDscMass];
  d->alpha0 = out[kDscAlpha0];
  d->peak = mx;
  d->hf_frac = out[kDscTot] > 0 ? out[kDscHF] / out[kDscTot] : 0.0;
  d->m2 = out[kDscM2] / (double)c->p.P;
  d->ring_radius = out[kDscRing] / (double)c->p.P;
  d->step = c->n;
  return SIPF_OK;
}

template <typename T> int upload_aos(sipf_ctx* c, const double* X) {
  const size_t bytes = (size_t)c->p.P * 3 * sizeof(double);
  double* stage = nullptr;
  SIPF_CK(cudaMalloc(&stage, bytes));
  cudaError_t e = cudaMemcpyAsync(stage, X, bytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = launch_aos_to_soa<T>(stage, c->p.P, make_geo<T>(c->p.L, c->p.H), (T*)c->st[0], (T*)c->st[1], (T*)c->st[2],
                             c->stream);
  if (e == cudaSuccess) e = launch_iota(c->st_id, c->p.P, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(stage);
  if (e != cudaSuccess) return cuda_fail(e, "upload positions");
  return rebin_from_staging<T>(c);
}

template <typename T> int positions_host(sipf_ctx* c, double* out) {
  const size_t P = (size_t)c->p.P;
  int r = unbin_to<T>(c, (T*)c->st[0], (T*)c->st[1], (T*)c->st[2]);
  if (r) return r;
  std::vector<T> h(3 * P);
  for (int d = 0; d < 3; ++d)
    SIPF_CK(cudaMemcpyAsync(h.data() + d * P, c->st[d], P * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < P; ++i)
    for (int d = 0; d < 3; ++d) out[3 * i + d] = (double)h[d * P + i];
  return SIPF_OK;
}

// Device addresses of three host buffers, when all three are page-locked
// allocations mapped into the device's address space (cudaHostAlloc /
// cudaHostRegister memory): kernels can then write them directly over the
// host link.  False for pageable memory (copies through the runtime instead).
bool host_device_views(const void* const h[3], void* d[3]) {
  for (int k = 0; k < 3; ++k) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h[k]) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return false;
    d[k] = at.devicePointer;
  }
  return true;
}

// Upload of host SoA positions.  With few enough tiles for the block-private
// re-bin, the positions are copied in pieces on the copy stream and each piece
// is wrapped and re-binned into the current buffer, with the current bin
// capacities, as soon as it has arrived (positions that do not fit a bin go to
// the overflow bin until the next capacity rebuild, at most resort_every
// steps later; results do not depend on the binning).  Otherwise: one copy,
// then the capacities are rebuilt from a tile histogram of the new positions.
template <typename T> int upload_soa_impl(sipf_ctx* c, const void* const src[3]) {
  const int64_t P = c->p.P;
  const Geo<T> g = make_geo<T>(c->p.L, c->p.H);
  if (c->NT > rebin_plain_max_tiles()) {
    for (int d = 0; d < 3; ++d)
      SIPF_CK(cudaMemcpyAsync(c->st[d], src[d], (size_t)P * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    SIPF_CK(launch_wrap_soa<T>(P, g, (T*)c->st[0], (T*)c->st[1], (T*)c->st[2], c->stream));
    SIPF_CK(launch_iota(c->st_id, P, c->stream));
    return rebin_from_staging<T>(c);
  }
  c->pos_ready = false;
  const int b = c->cur;
  SIPF_CK(cudaMemsetAsync(c->cursor[b], 0, (size_t)(c->NT + 1) * sizeof(int), c->stream));
  // the staging arrays are free once the context stream reaches this point
  SIPF_CK(cudaEventRecord(c->ev_begin, c->stream));
  SIPF_CK(cudaStreamWaitEvent(c->side[1], c->ev_begin, 0));
  const int np = pieces_for(P);
  for (int k = 0; k < np; ++k) {
    const int64_t a0 = piece_begin(P, np, k), a1 = piece_begin(P, np, k + 1);
    if (a1 <= a0) continue;
    for (int d = 0; d < 3; ++d)
      SIPF_CK(cudaMemcpyAsync((T*)c->st[d] + a0, (const T*)src[d] + a0, (size_t)(a1 - a0) * sizeof(T),
                              cudaMemcpyHostToDevice, c->side[1]));
    SIPF_CK(cudaEventRecord(c->ev_piece[k], c->side[1]));
    SIPF_CK(cudaStreamWaitEvent(c->stream, c->ev_piece[k], 0));
    cudaError_t e = cudaSuccess;
    launch_rebin_plain<T>((const T*)c->st[0] + a0, (const T*)c->st[1] + a0, (const T*)c->st[2] + a0, nullptr, a1 - a0,
                          g, c->shift, c->ntx, c->NT, (T*)c->bx[b][0], (T*)c->bx[b][1], (T*)c->bx[b][2], c->bid[b],
                          c->lbase[c->lc], c->lcap[c->lc], c->cursor[b], c->err, c->stream, &e, a0, true);
    SIPF_CK(e);
    c->launches += 1;
  }
  SIPF_CK(launch_chunk_list(cl_args(c, c->cursor[b], c->lcap[c->lc], c->lbase[c->lc], c->cursor[1 - b]), c->work,
                            nullptr, c->stream));
  c->launches += 2;
  SIPF_CK(mark_positions(c));
  c->dep_pending = true;
  return SIPF_OK;
}

// Download to host SoA positions.  Page-locked mapped buffers: a slot map
// of the current bins, then one kernel gathers the positions in id order and
// writes them straight into the host buffers (whole lines over the host
// link; no staging copy, no copy engine).  Otherwise on side streams as soon
// as the bins are final (the last step's deposit may still be running on the context
// stream): the bins' particles are partitioned by id into the copy's pieces
// (records in the other bin buffer), then each piece is scattered to particle
// order in the staging arrays and copied back, each piece's copy overlapping
// the next piece's scatter.  A piece's slots stay in L2 while its scattered
// sectors fill, where one scatter over all particles (16-byte records to
// random ids) wrote partial sectors to DRAM and had to finish before the
// first copy.
template <typename T> int download_soa_impl(sipf_ctx* c, void* const dst[3]) {
  const int64_t P = c->p.P;
  void* dv[3];
  if (c->cap_total <= (int64_t)UINT32_MAX && host_device_views(dst, dv)) {
    // page-locked mapped buffers: a slot map in the other buffer's id array
    // (free between steps), then the positions gathered in id order straight
    // into the host buffers, on the context stream
    SIPF_CK(cudaStreamWaitEvent(c->stream, c->ev_done, 0));   // a previous pieces download's copies
    SIPF_CK(launch_read_back_mapped<T>(bin_args<T>(c, c->cur, c->lc, -1, 0), c->max_chunks(), c->bid[1 - c->cur], P,
                                       (T*)dv[0], (T*)dv[1], (T*)dv[2], c->stream));
    c->launches += 2;
    return SIPF_OK;
  }
  // the other bin buffer is free between steps (the next move overwrites it)
  const int ob = 1 - c->cur;
  T* rx = (T*)c->bx[ob][0];
  T* ry = (T*)c->bx[ob][1];
  T* rz = (T*)c->bx[ob][2];
  uint32_t* rid = c->bid[ob];
  if (!c->pos_ready) SIPF_CK(mark_positions(c));
  SIPF_CK(cudaStreamWaitEvent(c->side[0], c->ev_pos, 0));
  SIPF_CK(cudaStreamWaitEvent(c->side[0], c->ev_done, 0));   // a previous download's copies
  const int np = pieces_for(P);
  PieceBounds pb{};
  pb.np = np;
  for (int k = 0; k <= np; ++k) pb.b[k] = piece_begin(P, np, k);
  SIPF_CK(cudaMemsetAsync(c->pcur, 0, PieceBounds::kMax * sizeof(int), c->side[0]));
  SIPF_CK(launch_partition_pieces<T>(bin_args<T>(c, c->cur, c->lc, -1, 0), c->max_chunks(), pb, c->pcur, rx, ry, rz,
                                     rid, c->side[0]));
  c->launches += 1;
  for (int k = 0; k < np; ++k) {
    const int64_t a0 = piece_begin(P, np, k), a1 = piece_begin(P, np, k + 1);
    if (a1 <= a0) continue;
    SIPF_CK(launch_scatter_piece<T>(rx, ry, rz, rid, a0, a1 - a0, P, (T*)c->st[0], (T*)c->st[1], (T*)c->st[2],
                                    c->side[0]));
    c->launches += 1;
    SIPF_CK(cudaEventRecord(c->ev_piece[k], c->side[0]));
    SIPF_CK(cudaStreamWaitEvent(c->side[1], c->ev_piece[k], 0));
    for (int d = 0; d < 3; ++d)
      SIPF_CK(cudaMemcpyAsync((T*)dst[d] + a0, (const T*)c->st[d] + a0, (size_t)(a1 - a0) * sizeof(T),
                              cudaMemcpyDeviceToHost, c->side[1]));
  }
  SIPF_CK(cudaEventRecord(c->ev_done, c->side[1]));
  SIPF_CK(cudaStreamWaitEvent(c->stream, c->ev_done, 0));
  return SIPF_OK;
}

template <typename T> int positions_dev_impl(sipf_ctx* c, void* x, void* y, void* z) {
  return unbin_to<T>(c, (T*)x, (T*)y, (T*)z);
}

template <typename T> int spectrum_host(sipf_ctx* c, double* out) {
  const size_t n = (size_t)c->S() * 2;
  std::vector<T> h(n);
  SIPF_CK(cudaMemcpyAsync(h.data(), c->alpha, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
  SIPF_CK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < n; ++i) out[i] = (double)h[i];
  return SIPF_OK;
}

void free_ctx(sipf_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (cudaStream_t t : c->side)
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  for (cudaEvent_t e : c->ev_piece)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->ev_pos, c->ev_begin, c->ev_done})
    if (e) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    for (int d = 0; d < 3; ++d) cudaFree(c->bx[b][d]);
    cudaFree(c->bid[b]);
    cudaFree(c->lcap[b]);
    cudaFree(c->lbase[b]);
    cudaFree(c->cursor[b]);
  }
  for (int d = 0; d < 3; ++d) cudaFree(c->st[d]);
  cudaFree(c->st_id);
  cudaFree(c->st_count);
  cudaFree(c->st_cap);
  cudaFree(c->st_base);
  cudaFree(c->count);
  cudaFree(c->chunk_start);
  cudaFree(c->chunks);
  cudaFree(c->part);
  cudaFree(c->work);
  cudaFree(c->ovf);
  cudaFree(c->hist);
  cudaFree(c->pcur);
  cudaFree(c->phi);
  cudaFree(c->T1);
  cudaFree(c->alpha);
  cudaFree(c->T2);
  cudaFree(c->grad);
  cudaFree(c->dsc);
  cudaFree(c->err);
  cudaFree(c->fft_run);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

#define DISPATCH(ctx, fn, ...) ((ctx)->p.precision == 64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

}  // namespace

extern "C" {

int sipf_params_default(sipf_params* p) {
  if (!p) return fail(SIPF_EINVAL, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->chi = p->mu = p->eps = p->k = 1.0;
  p->L = 1.0;
  p->mass = 1.0;
  p->dt = 1e-3;
  p->T = 0.0;
  p->H0 = -1.0;
  p->seed = 0;
  p->P = 0;
  p->H = 64;
  p->precision = 32;
  p->p2g_order = 4;
  p->g2p_order = 2;
  p->splitting = SIPF_SPLIT_HALF;
  p->deposit_mode = SIPF_DEPOSIT_ATOMIC;
  p->propagator = SIPF_PROP_IMPLICIT;
  p->resort_every = 0;
  return SIPF_OK;
}

int sipf_validate(const sipf_params* p) { return validate(p); }

int sipf_filter_scale(const sipf_params* p, double* H0_out) {
  if (!H0_out) return fail(SIPF_EINVAL, "H0_out is NULL");
  const int r = validate(p);
  if (r) return r;
  *H0_out = effective_H0(*p);
  return SIPF_OK;
}

int sipf_init(const sipf_params* p, const double* X0, void* stream, sipf_ctx** out) {
  if (!out) return fail(SIPF_EINVAL, "out is NULL");
  *out = nullptr;
  int r = validate(p);
  if (r) return r;
  if (!X0) return fail(SIPF_EINVAL, "X0 is NULL");
  for (int64_t i = 0; i < 3 * p->P; ++i)
    if (!isfinite(X0[i])) return fail(SIPF_ENONFINITE, "X0 holds a non-finite coordinate");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(SIPF_ENODEV, "no CUDA device");
  SIPF_CK(ensure_device_tables());
  sipf_ctx* c = new sipf_ctx();
  c->p = *p;
  c->H0 = effective_H0(*p);
  c->esz = p->precision == 64 ? 8 : 4;
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
    c->own_stream = true;
  }
  const size_t P = (size_t)p->P;
  const size_t N = (size_t)c->H3();
  const size_t S = (size_t)c->S();
  c->shift = binned_tile_shift(p->H);
  c->ntx = p->H <= 16 ? 1 : p->H >> c->shift;
  c->NT = c->ntx * c->ntx * c->ntx;
  const size_t nb = (size_t)c->NT + 1;
  // bins hold at most 1.5 P + 64 NT + 6 P / 4 (capacities with spare room), the overflow bin P
  c->cap_total = (int64_t)(4 * P + 68 * (size_t)c->NT + 1024);
  const size_t cap = (size_t)c->cap_total;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = cudaMalloc(&c->bx[b][d], cap * c->esz);
    if (e == cudaSuccess) e = cudaMalloc(&c->bid[b], cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->lcap[b], nb * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->lbase[b], nb * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->cursor[b], nb * sizeof(int));
  }
  // staging arrays padded to a multiple of 4 elements (16-byte bulk copies)
  const size_t P4 = (P + 3) & ~(size_t)3;
  for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = cudaMalloc(&c->st[d], P4 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->st_id, P4 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&c->st_count, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->st_cap, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->st_base, nb * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->count, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->chunk_start, (nb + 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->chunks, (size_t)c->max_chunks() * sizeof(ChunkDesc));
  if (e == cudaSuccess) e = cudaMalloc(&c->part, (size_t)chunk_list_blocks(c->NT) * sizeof(long long));
  // work counters: [0] deposit and re-bin passes, [1] the move (both cleared by
  // every chunk-list emission, so a step needs no separate clears)
  if (e == cudaSuccess) e = cudaMalloc(&c->work, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->work, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMalloc(&c->ovf, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ovf, 0, sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = cudaMalloc(&c->hist, nb * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->pcur, PieceBounds::kMax * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->phi, N * (c->fixed() ? 8 : c->esz));
  if (e == cudaSuccess) e = cudaMalloc(&c->T1, S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->alpha, S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->T2, 3 * S * 2 * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->grad, 4 * N * c->esz);
  if (e == cudaSuccess) e = cudaMalloc(&c->dsc, kDscCount * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->err, sizeof(int));
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking);
  for (int i = 0; i < sipf_ctx::kPieces && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&c->ev_piece[i], cudaEventDisableTiming);
  for (cudaEvent_t* ev : {&c->ev_pos, &c->ev_begin, &c->ev_done})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess && p->H >= 32) {
    e = cudaMalloc(&c->fft_run, p->precision == 64 ? sizeof(FftRun<double>) : sizeof(FftRun<float>));
    if (e == cudaSuccess) {
      if (p->precision == 64) {
        const FftRun<double> f = make_fft_run<double>(c);
        e = cudaMemcpy(c->fft_run, &f, sizeof(f), cudaMemcpyHostToDevice);
      } else {
        const FftRun<float> f = make_fft_run<float>(c);
        e = cudaMemcpy(c->fft_run, &f, sizeof(f), cudaMemcpyHostToDevice);
      }
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->alpha, 0, S * 2 * c->esz, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->dsc, 0, kDscCount * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->grad, 0, 4 * N * c->esz, c->stream);
  if (e == cudaSuccess) {
    // the staging described as one bin (the overflow slot) holding all P particles
    std::vector<int> cnt(nb, 0), capv(nb, 0);
    std::vector<long long> base(nb, 0);
    cnt[c->NT] = (int)P;
    capv[c->NT] = (int)P;
    e = cudaMemcpy(c->st_count, cnt.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->st_cap, capv.data(), nb * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->st_base, base.data(), nb * sizeof(long long), cudaMemcpyHostToDevice);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(c->cursor[b], 0, nb * sizeof(int), c->stream);
  }
  if (e != cudaSuccess) {
    free_ctx(c);
    return cuda_fail(e, "sipf_init allocation");
  }
  r = DISPATCH(c, upload_aos, c, X0);
  // X^(0) deposited now (Algorithm 4's initialisation), so phi is current for
  // callers that read the runs' grids directly (the batched form)
  if (!r) r = DISPATCH(c, flush_deposit, c);
  if (r) { free_ctx(c); return r; }
  *out = c;
  return SIPF_OK;
}

int sipf_step(sipf_ctx* c, int64_t nsteps) {
  if (!c) return fail(SIPF_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(SIPF_EINVAL, "nsteps < 0");
  if (c->n + nsteps > 0xFFFFFFFFLL) return fail(SIPF_EINVAL, "step counter would exceed 2^32 - 1");
  return DISPATCH(c, step_impl, c, nsteps);
}

int sipf_run(sipf_ctx* c) {
  if (!c) return fail(SIPF_EINVAL, "ctx is NULL");
  const int64_t NT = (int64_t)ceil(c->p.T / c->p.dt - 1e-9);
  return sipf_step(c, NT > c->n ? NT - c->n : 0);
}

int64_t sipf_current_step(const sipf_ctx* c) { return c ? c->n : -1; }

int sipf_positions(sipf_ctx* c, double* out) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, positions_host, c, out);
}

int sipf_set_positions(sipf_ctx* c, const double* X) {
  if (!c || !X) return fail(SIPF_EINVAL, "NULL argument");
  for (int64_t i = 0; i < 3 * c->p.P; ++i)
    if (!isfinite(X[i])) return fail(SIPF_ENONFINITE, "X holds a non-finite coordinate");
  return DISPATCH(c, upload_aos, c, X);
}

int sipf_upload_soa(sipf_ctx* c, const void* x, const void* y, const void* z) {
  if (!c || !x || !y || !z) return fail(SIPF_EINVAL, "NULL argument");
  const void* const src[3] = {x, y, z};
  return DISPATCH(c, upload_soa_impl, c, src);
}

int sipf_download_soa(sipf_ctx* c, void* x, void* y, void* z) {
  if (!c || !x || !y || !z) return fail(SIPF_EINVAL, "NULL argument");
  void* const dst[3] = {x, y, z};
  return DISPATCH(c, download_soa_impl, c, dst);
}

int sipf_positions_dev(sipf_ctx* c, void* x, void* y, void* z) {
  if (!c || !x || !y || !z) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, positions_dev_impl, c, x, y, z);
}

int sipf_density(sipf_ctx* c, double* out, int filtered) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, density_host, c, out, filtered);
}

int sipf_field(sipf_ctx* c, double* out) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, field_host, c, out);
}

int sipf_spectrum(sipf_ctx* c, double* out) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, spectrum_host, c, out);
}

int sipf_gradient(sipf_ctx* c, double* out) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, gradient_host, c, out);
}

int sipf_diagnostics(sipf_ctx* c, sipf_diag* d) {
  if (!c || !d) return fail(SIPF_EINVAL, "NULL argument");
  return DISPATCH(c, diagnostics_impl, c, d);
}

int sipf_sync(sipf_ctx* c) {
  if (!c) return fail(SIPF_EINVAL, "ctx is NULL");
  SIPF_CK(cudaStreamSynchronize(c->stream));
  int flag = 0;
  SIPF_CK(cudaMemcpy(&flag, c->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    SIPF_CK(cudaMemset(c->err, 0, sizeof(int)));
    if (flag & 1) return fail(SIPF_ENONFINITE, "a particle position became non-finite");
    if (flag & 4) return fail(SIPF_ETIMEOUT, "a bounded wait for a staging copy ran out");
    return fail(SIPF_ENOMEM, "the overflow bin of the particle layout was full");
  }
  return SIPF_OK;
}

void sipf_destroy(sipf_ctx* c) { free_ctx(c); }

int sipf_timing_enable(sipf_ctx* c, int enable) {
  if (!c) return fail(SIPF_EINVAL, "ctx is NULL");
  if (enable) {
    SIPF_CK(cudaStreamSynchronize(c->stream));
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    c->ev.clear();
    c->timed_steps = c->timed_kernels = 0;
    SIPF_CK(cudaMemsetAsync(c->ovf, 0, sizeof(unsigned long long), c->stream));
  }
  c->timing = enable != 0;
  return SIPF_OK;
}

int sipf_timing_read(sipf_ctx* c, sipf_timing* out) {
  if (!c || !out) return fail(SIPF_EINVAL, "NULL argument");
  SIPF_CK(cudaStreamSynchronize(c->stream));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (size_t i = 0; i + 7 <= c->ev.size(); i += 7)
    for (int k = 0; k < 6; ++k) {
      float ms = 0.f;
      SIPF_CK(cudaEventElapsedTime(&ms, c->ev[i + k], c->ev[i + k + 1]));
      acc[k] += ms;
    }
  // event order of a step: deposit, forward, spectral, inverse, move, bookkeeping
  out->deposit_ms = acc[0];
  out->forward_ms = acc[1];
  out->spectral_ms = acc[2];
  out->inverse_ms = acc[3];
  out->move_ms = acc[4];
  out->bookkeeping_ms = acc[5];
  out->steps = c->timed_steps;
  out->kernels = c->timed_kernels;
  unsigned long long ovf = 0;
  SIPF_CK(cudaMemcpy(&ovf, c->ovf, sizeof(ovf), cudaMemcpyDeviceToHost));
  out->overflow = (int64_t)ovf;
  return SIPF_OK;
}

int64_t sipf_kernel_launches(const sipf_ctx* c) { return c ? c->launches : -1; }

const char* sipf_strerror(int code) {
  switch (code) {
    case SIPF_OK: return "ok";
    case SIPF_EINVAL: return "invalid argument";
    case SIPF_ENOMEM: return "out of memory";
    case SIPF_ECUDA: return "CUDA error";
    case SIPF_ENONFINITE: return "non-finite value";
    case SIPF_ETIMEOUT: return "device wait timed out";
    case SIPF_ENODEV: return "no CUDA device";
  }
  return "unknown error";
}

const char* sipf_last_error(void) { return g_last_error.c_str(); }

// ---- stateless operators ------------------------------------------------------

int sipf_noise_dev(int precision, uint64_t seed, int64_t step, int64_t first, int64_t P, void* z, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (P < 0 || first < 0 || step < 0 || step > 0xFFFFFFFFLL || (!z && P > 0)) return fail(SIPF_EINVAL, "noise args");
  if (P == 0) return SIPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  SIPF_CK(precision == 64 ? launch_noise<double>(seed, step, first, P, (double*)z, s)
                          : launch_noise<float>(seed, step, first, P, (float*)z, s));
  return SIPF_OK;
}

int sipf_deposit_dev(int precision, const void* x, const void* y, const void* z, int64_t P, int32_t H, double L,
                     double w, int32_t order, void* grid, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (!is_pow2(H) || H < 8 || H > kNmax || !(L > 0) || P < 0 || (order != 2 && order != 4) || !grid)
    return fail(SIPF_EINVAL, "deposit args");
  if (P > 0 && (!x || !y || !z)) return fail(SIPF_EINVAL, "NULL positions");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)H * H * H;
  SIPF_CK(cudaMemsetAsync(grid, 0, N * (precision == 64 ? 8 : 4), s));
  if (P == 0) return SIPF_OK;
  if (precision == 64)
    SIPF_CK(launch_deposit<double>((const double*)x, (const double*)y, (const double*)z, P, make_geo<double>(L, H),
                                   w, (double*)grid, order, s));
  else
    SIPF_CK(launch_deposit<float>((const float*)x, (const float*)y, (const float*)z, P, make_geo<float>(L, H),
                                  (float)w, (float*)grid, order, s));
  return SIPF_OK;
}

int sipf_gather_dev(int precision, const void* x, const void* y, const void* z, int64_t P, int32_t H, double L,
                    const void* f, int32_t ncomp, int32_t order, void* out, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (!is_pow2(H) || H < 8 || H > kNmax || !(L > 0) || P < 0 || (order != 2 && order != 4) || !f || ncomp < 1 ||
      ncomp > 16)
    return fail(SIPF_EINVAL, "gather args");
  if (P == 0) return SIPF_OK;
  if (!x || !y || !z || !out) return fail(SIPF_EINVAL, "NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == 64)
    SIPF_CK(launch_gather<double>((const double*)x, (const double*)y, (const double*)z, P, make_geo<double>(L, H),
                                  (const double*)f, ncomp, order, (double*)out, s));
  else
    SIPF_CK(launch_gather<float>((const float*)x, (const float*)y, (const float*)z, P, make_geo<float>(L, H),
                                 (const float*)f, ncomp, order, (float*)out, s));
  return SIPF_OK;
}

int sipf_forward_ft_dev(int precision, int32_t H, double L, const void* grid, void* spec, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (!is_pow2(H) || H < 8 || H > kNmax || !(L > 0) || !grid || !spec) return fail(SIPF_EINVAL, "forward_ft args");
  SIPF_CK(ensure_device_tables());
  cudaStream_t s = (cudaStream_t)stream;
  const int nh = H / 2 + 1;
  const double sc = 1.0 / (L * L * L);
  if (precision == 64) {
    cpx<double>* o = (cpx<double>*)spec;
    SIPF_CK(launch_rows_r2c<double>(grid, 0, 1.0, false, o, H, H * H, nullptr, s));
    SIPF_CK(launch_cols<double>(o, H, H, nh, 1, 0, -1, 1.0, s));
    SIPF_CK(launch_cols<double>(o, H, 1, H * nh, 1, 0, -1, sc, s));
  } else {
    cpx<float>* o = (cpx<float>*)spec;
    SIPF_CK(launch_rows_r2c<float>(grid, 0, 1.0, false, o, H, H * H, nullptr, s));
    SIPF_CK(launch_cols<float>(o, H, H, nh, 1, 0, -1, 1.0, s));
    SIPF_CK(launch_cols<float>(o, H, 1, H * nh, 1, 0, -1, sc, s));
  }
  return SIPF_OK;
}

int sipf_inverse_ft_dev(int precision, int32_t H, void* spec, void* grid, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (!is_pow2(H) || H < 8 || H > kNmax || !grid || !spec) return fail(SIPF_EINVAL, "inverse_ft args");
  SIPF_CK(ensure_device_tables());
  cudaStream_t s = (cudaStream_t)stream;
  const int nh = H / 2 + 1;
  if (precision == 64) {
    cpx<double>* o = (cpx<double>*)spec;
    SIPF_CK(launch_cols<double>(o, H, 1, H * nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_cols<double>(o, H, H, nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_rows_c2r<double>(o, 1, 0, (double*)grid, H, H * H, nullptr, s));
  } else {
    cpx<float>* o = (cpx<float>*)spec;
    SIPF_CK(launch_cols<float>(o, H, 1, H * nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_cols<float>(o, H, H, nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_rows_c2r<float>(o, 1, 0, (float*)grid, H, H * H, nullptr, s));
  }
  return SIPF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Inverse transform that allocates nothing.
//
// Its work space is the file-scope array below, sized for one half spectrum
// of H = 64 in double precision; every GPU that loads the library holds these
// bytes until the process exits.  Host code must not use the array's name as
// a device address: the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocMaxH = 64;
static constexpr size_t kNoAllocScratchBytes = kNoAllocMaxH * kNoAllocMaxH * (kNoAllocMaxH / 2 + 1) * 2 * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

int noalloc_scratch(void** out) {
  int dev = 0;
  SIPF_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SIPF_EINVAL, "device index beyond the supported range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    SIPF_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SIPF_OK;
}
}  // namespace

extern "C" int sipf_inverse_ft_noalloc_dev(int precision, int32_t H, const void* spec, void* grid, void* stream) {
  if (precision != 32 && precision != 64) return fail(SIPF_EINVAL, "precision");
  if (!is_pow2(H) || H < 8 || H > kNmax || !grid || !spec) return fail(SIPF_EINVAL, "inverse_ft_noalloc args");
  const size_t nh = (size_t)H / 2 + 1;
  const size_t bytes = (size_t)H * H * nh * 2 * (precision == 64 ? 8 : 4);
  if (bytes > kNoAllocScratchBytes)
    return fail(SIPF_EINVAL, "sipf_inverse_ft_noalloc_dev: the spectrum (" + std::to_string(bytes) +
                                 " bytes) exceeds the built-in work space of " + std::to_string(kNoAllocScratchBytes) +
                                 " bytes (H <= 64)");
  SIPF_CK(ensure_device_tables());
  void* work = nullptr;
  int r = noalloc_scratch(&work);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  SIPF_CK(cudaMemcpyAsync(work, spec, bytes, cudaMemcpyDeviceToDevice, s));
  if (precision == 64) {
    cpx<double>* o = (cpx<double>*)work;
    SIPF_CK(launch_cols<double>(o, H, 1, H * (int)nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_cols<double>(o, H, H, (int)nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_rows_c2r<double>(o, 1, 0, (double*)grid, H, H * H, nullptr, s));
  } else {
    cpx<float>* o = (cpx<float>*)work;
    SIPF_CK(launch_cols<float>(o, H, 1, H * (int)nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_cols<float>(o, H, H, (int)nh, 1, 0, +1, 1.0, s));
    SIPF_CK(launch_rows_c2r<float>(o, 1, 0, (float*)grid, H, H * H, nullptr, s));
  }
  return SIPF_OK;
}

// ===========================================================================
// Batched runs: independent SIPF-PIC runs of uneven P, H, chi, seed, ... in
// the same launches.  Each run keeps the state of an ordinary context; the
// batch issues, per step, the field solve once per grid size (runs of equal
// H share each launch) and the particle passes once for all runs (work items
// of all runs from one counter).  Steps are captured in CUDA graphs of 32
// steps, the period after which the buffer and layout parities repeat; the
// step counter lives in device memory so the graph can be replayed.
// ===========================================================================
struct sipf_batch {
  int nruns = 0;
  std::vector<sipf_ctx*> runs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int precision = 32;
  bool fixed = false;
  int g2p = 0;   // the gather order shared by all runs (2 or 4), 0 if they differ
  std::vector<int> group_H, group_n;
  std::vector<void*> fft_tab;                    // device FftRun<T>[group_n]
  void* move_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  void* rebin_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  void* dep_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  ChunkListArgs* cl_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  LayoutArgs* ly_tab[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  long long* prefix = nullptr;
  unsigned long long* work = nullptr;
  uint32_t* step = nullptr;
  int cur = 0, lc = 1, since = 0;
  int64_t n = 0;
  bool use_graph = true;
  cudaGraphExec_t graph = nullptr;
  int graph_cur = -1, graph_lc = -1, graph_since = -1;
  int64_t launches = 0;
  int max_NT = 1;   // most tiles of any run (grid of the batched chunk-list passes)
  int field_kernels = 0;   // field-solve kernels of the last issued step
  // launch shapes (autotuned) and per-phase events of the last issued step
  std::vector<FieldTune> field_tune;
  int move_bps = 0, dep_bps = 0;
  bool record_phases = false;
  std::vector<cudaEvent_t> ev;   // 2 per group, then move pair, deposit pair
};

namespace {

constexpr int kBatchResort = 16;
constexpr int kBatchGraphSteps = 32;
constexpr int kBatchMaxRuns = 4096;   // 3 x runs block rows of the inverse y pass stay below 65535

void batch_free(sipf_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->fft_tab) cudaFree(p);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      cudaFree(b->move_tab[i][j]);
      cudaFree(b->rebin_tab[i][j]);
      cudaFree(b->dep_tab[i][j]);
      cudaFree(b->cl_tab[i][j]);
      cudaFree(b->ly_tab[i][j]);
    }
  cudaFree(b->prefix);
  cudaFree(b->work);
  cudaFree(b->step);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  for (sipf_ctx* c : b->runs) free_ctx(c);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

template <typename T> int batch_tables(sipf_batch* b) {
  const int R = b->nruns;
  // field-solve tables per grid size
  for (int g = 0; g < (int)b->group_H.size(); ++g) {
    std::vector<FftRun<T>> t;
    for (sipf_ctx* c : b->runs) {
      if (c->p.H != b->group_H[g]) continue;
      const FftRun<T> f = make_fft_run<T>(c);
      t.push_back(f);
    }
    void* d = nullptr;
    SIPF_CK(cudaMalloc(&d, t.size() * sizeof(FftRun<T>)));
    b->fft_tab.push_back(d);
    SIPF_CK(cudaMemcpy(d, t.data(), t.size() * sizeof(FftRun<T>), cudaMemcpyHostToDevice));
  }
  // particle tables for every (buffer, layout) parity
  for (int cur = 0; cur < 2; ++cur)
    for (int lc = 0; lc < 2; ++lc) {
      std::vector<BinArgs<T>> mv, rb, dp;
      std::vector<ChunkListArgs> cl;
      std::vector<LayoutArgs> ly;
      for (sipf_ctx* c : b->runs) {
        mv.push_back(bin_args<T>(c, cur, lc, 1 - cur, lc));
        rb.push_back(bin_args<T>(c, cur, lc, 1 - cur, 1 - lc));
        dp.push_back(bin_args<T>(c, cur, lc, -1, 0));
        // chunk list of buffer `cur` written with layout `lc`
        cl.push_back(cl_args(c, c->cursor[cur], c->lcap[lc], c->lbase[lc], c->cursor[1 - cur]));
        // new layout `lc` from the counts of buffer `cur`
        ly.push_back(LayoutArgs{c->cursor[cur], c->lcap[lc], c->lbase[lc], c->NT, c->ntx, (int)c->p.P});
      }
      SIPF_CK(cudaMalloc(&b->move_tab[cur][lc], R * sizeof(BinArgs<T>)));
      SIPF_CK(cudaMalloc(&b->rebin_tab[cur][lc], R * sizeof(BinArgs<T>)));
      SIPF_CK(cudaMalloc(&b->dep_tab[cur][lc], R * sizeof(BinArgs<T>)));
      SIPF_CK(cudaMalloc(&b->cl_tab[cur][lc], R * sizeof(ChunkListArgs)));
      SIPF_CK(cudaMalloc(&b->ly_tab[cur][lc], R * sizeof(LayoutArgs)));
      SIPF_CK(cudaMemcpy(b->move_tab[cur][lc], mv.data(), R * sizeof(BinArgs<T>), cudaMemcpyHostToDevice));
      SIPF_CK(cudaMemcpy(b->rebin_tab[cur][lc], rb.data(), R * sizeof(BinArgs<T>), cudaMemcpyHostToDevice));
      SIPF_CK(cudaMemcpy(b->dep_tab[cur][lc], dp.data(), R * sizeof(BinArgs<T>), cudaMemcpyHostToDevice));
      SIPF_CK(cudaMemcpy(b->cl_tab[cur][lc], cl.data(), R * sizeof(ChunkListArgs), cudaMemcpyHostToDevice));
      SIPF_CK(cudaMemcpy(b->ly_tab[cur][lc], ly.data(), R * sizeof(LayoutArgs), cudaMemcpyHostToDevice));
    }
  return SIPF_OK;
}

// Enqueue one step of every run (mirrors step_impl) and advance the host-side
// parities.
template <typename T> int batch_issue_step(sipf_batch* b) {
  const int R = b->nruns;
  cudaStream_t s = b->stream;
  const int G = (int)b->group_H.size();
  int fk = 0;   // field-solve kernels launched this step
  auto mark = [&](int i) -> cudaError_t { return b->record_phases ? cudaEventRecord(b->ev[i], s) : cudaSuccess; };
  for (int g = 0; g < G; ++g) {
    SIPF_CK(mark(2 * g));
    SIPF_CK(launch_field_batch<T>((const FftRun<T>*)b->fft_tab[g], b->group_n[g], b->group_H[g], kFieldAll, s,
                                  b->field_tune[g], &fk));
    SIPF_CK(mark(2 * g + 1));
  }
  SIPF_CK(mark(2 * G));
  SIPF_CK(cudaMemsetAsync(b->work, 0, sizeof(unsigned long long), s));
  SIPF_CK(launch_move_batch<T>((const BinArgs<T>*)b->move_tab[b->cur][b->lc], b->prefix, R, b->work, b->step, true, s,
                               b->move_bps, b->g2p));
  SIPF_CK(launch_chunk_list_batch(b->cl_tab[1 - b->cur][b->lc], R, b->max_NT, s));
  SIPF_CK(launch_run_prefix(b->cl_tab[1 - b->cur][b->lc], R, b->prefix, b->work, b->step, 1, s));
  SIPF_CK(mark(2 * G + 1));
  b->launches += fk + 4;
  b->field_kernels = fk;
  b->cur = 1 - b->cur;
  if (++b->since >= kBatchResort) {
    SIPF_CK(launch_layout_batch(b->ly_tab[b->cur][1 - b->lc], R, s));
    SIPF_CK(launch_move_batch<T>((const BinArgs<T>*)b->rebin_tab[b->cur][b->lc], b->prefix, R, b->work, b->step, false,
                                 s, b->move_bps));
    SIPF_CK(launch_chunk_list_batch(b->cl_tab[1 - b->cur][1 - b->lc], R, b->max_NT, s));
    SIPF_CK(launch_run_prefix(b->cl_tab[1 - b->cur][1 - b->lc], R, b->prefix, b->work, b->step, 0, s));
    b->launches += 5;
    b->cur = 1 - b->cur;
    b->lc = 1 - b->lc;
    b->since = 0;
  }
  SIPF_CK(mark(2 * G + 2));
  SIPF_CK(launch_deposit_batch<T>((const BinArgs<T>*)b->dep_tab[b->cur][b->lc], b->prefix, R, b->work, b->fixed, s,
                                  b->dep_bps));
  SIPF_CK(mark(2 * G + 3));
  b->launches += 1;
  b->n += 1;
  return SIPF_OK;
}

template <typename T> int batch_step_impl(sipf_batch* b, int64_t nsteps) {
  while (nsteps > 0) {
    if (b->use_graph && nsteps >= kBatchGraphSteps) {
      if (!b->graph || b->graph_cur != b->cur || b->graph_lc != b->lc || b->graph_since != b->since) {
        if (b->graph) {
          cudaGraphExecDestroy(b->graph);
          b->graph = nullptr;
        }
        const int c0 = b->cur, l0 = b->lc, s0 = b->since;
        const int64_t n0 = b->n, k0 = b->launches;
        SIPF_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        int r = SIPF_OK;
        for (int i = 0; i < kBatchGraphSteps && r == SIPF_OK; ++i) r = batch_issue_step<T>(b);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (r) {
          if (g) cudaGraphDestroy(g);
          return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        const cudaError_t e2 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate");
        // capture issued nothing: restore the parities, they advance on launch
        b->cur = c0;
        b->lc = l0;
        b->since = s0;
        b->n = n0;
        b->launches = k0;
        b->graph_cur = c0;
        b->graph_lc = l0;
        b->graph_since = s0;
      }
      SIPF_CK(cudaGraphLaunch(b->graph, b->stream));
      // 32 steps hold 32 moves and 2 capacity rebuilds: parities return
      b->n += kBatchGraphSteps;
      b->launches += kBatchGraphSteps * ((int64_t)b->field_kernels + 5) + 2 * 5;
      nsteps -= kBatchGraphSteps;
    } else {
      int r = batch_issue_step<T>(b);
      if (r) return r;
      nsteps -= 1;
    }
  }
  return SIPF_OK;
}

// Autotuner: coordinate descent over the launch shapes, each candidate timed
// on real steps of the batch (the first step of a trial warms the shapes, the
// fastest of the others counts).  Shapes do not change results, so the runs
// simply advance by the steps spent here.
template <typename T> int batch_autotune_impl(sipf_batch* b, int trial, sipf_batch_tuning* out) {
  const int G = (int)b->group_H.size();
  const int64_t n0 = b->n;
  b->record_phases = true;
  auto measure = [&](int e0, int e1, float* ms) -> int {
    float best = 3.0e38f;
    for (int i = 0; i < trial; ++i) {
      int r = batch_issue_step<T>(b);
      if (r) return r;
      if (i == 0) continue;
      SIPF_CK(cudaEventSynchronize(b->ev[e1]));
      float t = 0.f;
      SIPF_CK(cudaEventElapsedTime(&t, b->ev[e0], b->ev[e1]));
      best = std::min(best, t);
    }
    *ms = best;
    return SIPF_OK;
  };
  std::vector<float> field_ms(G, 0.f);
  for (int g = 0; g < G; ++g) {
    FieldTune best_t = field_tune_default<T>(b->group_H[g]);
    float best = 3.0e38f;
    // plane kernels or pencil passes first, then the x-pass tile, then the
    // pencil-pass shapes (which only matter if pencils won)
    static const std::vector<int> cand[7] = {{0, 1, 2}, {8, 16, 32}, {1, 2}, {4, 8, 16}, {8, 16}, {8, 16, 32}, {4, 8, 16}};
    for (int dim = 0; dim < 7; ++dim) {
      for (int v : cand[dim]) {
        FieldTune t = best_t;
        int* f[7] = {&t.plane_mode, &t.plane_nw, &t.inv3, &t.sbc, &t.spec_nw, &t.bc, &t.rows_per_sm};
        *f[dim] = v;
        if (!field_tune_valid<T>(b->group_H[g], t)) continue;
        b->field_tune[g] = t;
        float ms = 0.f;
        int r = measure(2 * g, 2 * g + 1, &ms);
        if (r) return r;
        if (ms < best) {
          best = ms;
          best_t = t;
        }
      }
      b->field_tune[g] = best_t;
    }
    field_ms[g] = best;
  }
  float move_ms = 3.0e38f, dep_ms = 3.0e38f;
  {
    int best_c = b->move_bps;
    for (int c : {1, 2, 3, 0}) {
      b->move_bps = c;
      float ms = 0.f;
      int r = measure(2 * G, 2 * G + 1, &ms);
      if (r) return r;
      if (ms < move_ms) {
        move_ms = ms;
        best_c = c;
      }
    }
    b->move_bps = best_c;
  }
  {
    int best_c = b->dep_bps;
    for (int c : {1, 2, 3, 4, 0}) {
      b->dep_bps = c;
      float ms = 0.f;
      int r = measure(2 * G + 2, 2 * G + 3, &ms);
      if (r) return r;
      if (ms < dep_ms) {
        dep_ms = ms;
        best_c = c;
      }
    }
    b->dep_bps = best_c;
  }
  b->record_phases = false;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    out->ngroups = G;
    for (int g = 0; g < G && g < 4; ++g) {
      out->H[g] = b->group_H[g];
      out->cols_tile[g] = b->field_tune[g].bc;
      out->xpass_tile[g] = b->field_tune[g].sbc;
      out->rows_blocks_per_sm[g] = b->field_tune[g].rows_per_sm;
      const int pm = b->field_tune[g].plane_mode;
      out->plane_kernels[g] = pm == 0 ? 1 : (pm == 1 ? 0 : 2);
      out->plane_warps[g] = b->field_tune[g].plane_nw;
      out->xpass_warps[g] = b->field_tune[g].spec_nw;
      out->inverse_all_components[g] = b->field_tune[g].inv3;
      out->field_ms[g] = field_ms[g];
    }
    out->move_blocks_per_sm = b->move_bps;
    out->deposit_blocks_per_sm = b->dep_bps;
    out->move_ms = move_ms;
    out->deposit_ms = dep_ms;
    out->steps_used = b->n - n0;
  }
  return SIPF_OK;
}

// Make run r's context describe the batch's current state.
void batch_sync_run(sipf_batch* b, int r) {
  sipf_ctx* c = b->runs[r];
  c->cur = b->cur;
  c->lc = b->lc;
  c->n = b->n;
  c->since_layout = b->since;
}

}  // namespace

extern "C" {

int sipf_batch_init(int32_t nruns, const sipf_params* params, const double* const* X0, void* stream,
                    sipf_batch** out) {
  if (!out) return fail(SIPF_EINVAL, "out is NULL");
  *out = nullptr;
  if (nruns < 1 || !params || !X0) return fail(SIPF_EINVAL, "batch needs nruns >= 1, params and X0");
  if (nruns > kBatchMaxRuns) return fail(SIPF_EINVAL, "batch holds at most 4096 runs");
  for (int r = 0; r < nruns; ++r) {
    const sipf_params& p = params[r];
    int v = validate(&p);
    if (v) return fail(v, "run " + std::to_string(r) + ": " + g_last_error);
    if (p.H < 32) return fail(SIPF_EINVAL, "run " + std::to_string(r) + ": batched runs need H >= 32");
    if (p.precision != params[0].precision || p.deposit_mode != params[0].deposit_mode)
      return fail(SIPF_EINVAL, "run " + std::to_string(r) + ": precision and deposit_mode must match run 0");
    if (p.resort_every != 0 && p.resort_every != kBatchResort)
      return fail(SIPF_EINVAL, "run " + std::to_string(r) + ": batched runs rebuild capacities every 16 steps");
    if (!X0[r]) return fail(SIPF_EINVAL, "run " + std::to_string(r) + ": X0 is NULL");
  }
  sipf_batch* b = new sipf_batch();
  b->nruns = nruns;
  b->precision = params[0].precision;
  b->fixed = params[0].deposit_mode == SIPF_DEPOSIT_DETERMINISTIC;
  b->g2p = params[0].g2p_order;
  for (int r = 1; r < nruns; ++r)
    if (params[r].g2p_order != b->g2p) b->g2p = 0;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return cuda_fail(e, "cudaStreamCreate");
    }
    b->own_stream = true;
  }
  for (int r = 0; r < nruns; ++r) {
    sipf_ctx* c = nullptr;
    int v = sipf_init(&params[r], X0[r], b->stream, &c);
    if (v) {
      batch_free(b);
      return v;
    }
    b->runs.push_back(c);
    // many sparse runs: merge windows of 16 bins; the current bins' chunk
    // list is made again with them (their counts are unchanged)
    c->merge = 16;
    cudaError_t e = launch_chunk_list(cl_args(c, c->cursor[c->cur], c->lcap[c->lc], c->lbase[c->lc],
                                              c->cursor[1 - c->cur]),
                                      c->work, nullptr, c->stream);
    if (e != cudaSuccess) {
      batch_free(b);
      return cuda_fail(e, "sipf_batch_init chunk list");
    }
  }
  for (sipf_ctx* c : b->runs) {
    bool found = false;
    for (size_t g = 0; g < b->group_H.size(); ++g)
      if (b->group_H[g] == c->p.H) {
        b->group_n[g] += 1;
        found = true;
      }
    if (!found) {
      b->group_H.push_back(c->p.H);
      b->group_n.push_back(1);
    }
  }
  b->field_tune.assign(b->group_H.size(), FieldTune{});
  for (sipf_ctx* c : b->runs) b->max_NT = std::max(b->max_NT, c->NT);
  cudaError_t e = cudaMalloc(&b->prefix, (nruns + 1) * sizeof(long long));
  for (size_t i = 0; i < 2 * b->group_H.size() + 4 && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreate(&ev);
    if (e == cudaSuccess) b->ev.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->work, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->step, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->step, 0, sizeof(uint32_t), b->stream);
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "sipf_batch_init allocation");
  }
  b->cur = b->runs[0]->cur;
  b->lc = b->runs[0]->lc;
  int r = b->precision == 64 ? batch_tables<double>(b) : batch_tables<float>(b);
  if (!r) {
    cudaError_t e3 = launch_run_prefix(b->cl_tab[b->cur][b->lc], nruns, b->prefix, b->work, b->step, 0, b->stream);
    if (e3 == cudaSuccess) e3 = cudaStreamSynchronize(b->stream);
    if (e3 != cudaSuccess) r = cuda_fail(e3, "sipf_batch_init prefix");
  }
  if (r) {
    batch_free(b);
    return r;
  }
  *out = b;
  return SIPF_OK;
}

int sipf_batch_step(sipf_batch* b, int64_t nsteps) {
  if (!b) return fail(SIPF_EINVAL, "batch is NULL");
  if (nsteps < 0) return fail(SIPF_EINVAL, "nsteps < 0");
  if (b->n + nsteps > 0xFFFFFFFFLL) return fail(SIPF_EINVAL, "step counter would exceed 2^32 - 1");
  return b->precision == 64 ? batch_step_impl<double>(b, nsteps) : batch_step_impl<float>(b, nsteps);
}

int sipf_batch_autotune(sipf_batch* b, int32_t steps_per_trial, sipf_batch_tuning* out) {
  if (!b) return fail(SIPF_EINVAL, "batch is NULL");
  if (steps_per_trial < 2) return fail(SIPF_EINVAL, "steps_per_trial (>= 2)");
  const int64_t most = (int64_t)steps_per_trial * (18 * (int64_t)b->group_H.size() + 9);
  if (b->n + most > 0xFFFFFFFFLL) return fail(SIPF_EINVAL, "step counter would exceed 2^32 - 1");
  int r = b->precision == 64 ? batch_autotune_impl<double>(b, steps_per_trial, out)
                             : batch_autotune_impl<float>(b, steps_per_trial, out);
  b->record_phases = false;
  return r;
}

int sipf_batch_set_tuning(sipf_batch* b, const sipf_batch_tuning* t) {
  if (!b || !t) return fail(SIPF_EINVAL, "batch or tuning is NULL");
  if (t->ngroups != (int)b->group_H.size()) return fail(SIPF_EINVAL, "tuning has a different number of H groups");
  std::vector<FieldTune> ft(b->group_H.size());
  for (size_t g = 0; g < ft.size(); ++g) {
    if (t->H[g] != b->group_H[g]) return fail(SIPF_EINVAL, "tuning groups are in a different H order");
    ft[g].bc = t->cols_tile[g];
    ft[g].sbc = t->xpass_tile[g];
    ft[g].rows_per_sm = t->rows_blocks_per_sm[g];
    ft[g].plane_mode = t->plane_kernels[g] == 2 ? 2 : (t->plane_kernels[g] ? 0 : 1);
    ft[g].plane_nw = t->plane_warps[g];
    ft[g].spec_nw = t->xpass_warps[g];
    ft[g].inv3 = t->inverse_all_components[g];
    const bool ok = b->precision == 64 ? field_tune_valid<double>(b->group_H[g], ft[g])
                                       : field_tune_valid<float>(b->group_H[g], ft[g]);
    if (!ok) return fail(SIPF_EINVAL, "tuning group " + std::to_string(g) + " has an unsupported tile shape");
  }
  if (t->move_blocks_per_sm < 0 || t->move_blocks_per_sm > 32 || t->deposit_blocks_per_sm < 0 ||
      t->deposit_blocks_per_sm > 32)
    return fail(SIPF_EINVAL, "blocks per SM (0..32)");
  b->field_tune = ft;
  b->move_bps = t->move_blocks_per_sm;
  b->dep_bps = t->deposit_blocks_per_sm;
  if (b->graph) {
    SIPF_CK(cudaStreamSynchronize(b->stream));
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return SIPF_OK;
}

int sipf_batch_use_graph(sipf_batch* b, int enable) {
  if (!b) return fail(SIPF_EINVAL, "batch is NULL");
  b->use_graph = enable != 0;
  return SIPF_OK;
}

int64_t sipf_batch_current_step(const sipf_batch* b) { return b ? b->n : -1; }

int64_t sipf_batch_kernel_launches(const sipf_batch* b) { return b ? b->launches : -1; }

int sipf_batch_positions(sipf_batch* b, int32_t run, double* out) {
  if (!b || !out || run < 0 || run >= b->nruns) return fail(SIPF_EINVAL, "bad batch, run or out");
  batch_sync_run(b, run);
  return sipf_positions(b->runs[run], out);
}

int sipf_batch_diagnostics(sipf_batch* b, int32_t run, sipf_diag* out) {
  if (!b || !out || run < 0 || run >= b->nruns) return fail(SIPF_EINVAL, "bad batch, run or out");
  batch_sync_run(b, run);
  return sipf_diagnostics(b->runs[run], out);
}

int sipf_batch_spectrum(sipf_batch* b, int32_t run, double* out) {
  if (!b || !out || run < 0 || run >= b->nruns) return fail(SIPF_EINVAL, "bad batch, run or out");
  batch_sync_run(b, run);
  return sipf_spectrum(b->runs[run], out);
}

int sipf_batch_sync(sipf_batch* b) {
  if (!b) return fail(SIPF_EINVAL, "batch is NULL");
  SIPF_CK(cudaStreamSynchronize(b->stream));
  for (sipf_ctx* c : b->runs) {
    int r = sipf_sync(c);
    if (r) return r;
  }
  return SIPF_OK;
}

void sipf_batch_destroy(sipf_batch* b) { batch_free(b); }

}  // extern "C"

// ===========================================================================
// Adjoint form: gradients of a function of rho(T) with respect to chi, mu and
// X^0 through N steps of Algorithm 4 with the noise held fixed.  The forward
// pass keeps (X^n in id order, alpha^n) every `C` steps; the reverse sweep
// recomputes one segment of C steps at a time from its checkpoint, storing
// X^{n-1} and the gradient grids g^{n-1} of each step, and runs the
// transposed operators backwards through it.
// ===========================================================================
struct sipf_adjoint {
  sipf_ctx* c = nullptr;
  int64_t N = 0;
  int C = 20;
  int nck = 0;
  void* ckX = nullptr;     // nck x 3P T: X^{kC} (x plane, y plane, z plane)
  void* ckA = nullptr;     // nck x S complex T: alpha^{kC}
  void* segX = nullptr;    // C x 3P T: X^{n-1} of the segment being reversed, in bin order (x, y, z planes)
  uint32_t* segI = nullptr;  // C x P: the particle id of each segX entry
  void* segG = nullptr;    // C x 4 H^3 T: g^{n-1} as (gx, gy, gz, 0) nodes
  void* XN = nullptr;      // 3P T: X^N
  void* xb = nullptr;      // 4P T: Xbar as (x, y, z, 0) per particle
  unsigned long long* cursor = nullptr;   // scratch of the bin-order copies
  void* abar = nullptr;    // S complex T
  void* spec = nullptr;    // S complex T: L^-3 B abar, then inverse-transform work
  void* gbar = nullptr;    // 3 H^3 T: cotangent planes (the transforms' input)
  void* gbar4 = nullptr;   // 4 H^3 T: cotangents accumulated as (x, y, z, -) nodes, kept zero between steps
  void* ghat = nullptr;    // 3 S complex T
  void* phibar = nullptr;  // H^3 T
  void* phibar4 = nullptr; // 4 H^3 T: z-quads of phibar (the reverse step's Gamma_4 transpose reads them)
  void* fwd_tab = nullptr; // H >= 32: three FftRun<T> (cotangent plane d -> ghat d) for the plane forward transforms
  double* acc = nullptr;   // [dJ/dchi, dJ/ds]
  std::vector<double> X0;
  bool have_forward = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t launches = 0;    // adjoint kernels (the forward steps count in the context)
};

namespace {

constexpr int kAdjCheckpoint = 20;

void adjoint_free(sipf_adjoint* a) {
  if (!a) return;
  if (a->c && a->c->stream) cudaStreamSynchronize(a->c->stream);
  for (void* p : {a->ckX, a->ckA, a->segX, (void*)a->segI, a->segG, a->XN, a->xb, a->abar, a->spec, a->gbar,
                  a->gbar4, a->ghat, a->phibar, a->phibar4, (void*)a->cursor, a->fwd_tab})
    cudaFree(p);
  cudaFree(a->acc);
  for (cudaEvent_t e : a->ev)
    if (e) cudaEventDestroy(e);
  free_ctx(a->c);
  delete a;
}

// The three cotangent planes as runs of the batched field-solve kernels, so
// their forward transforms (rows r2c and the y axis) run as one plane kernel
// launch (H >= 32); the plane kernel clears each plane as it reads it.
template <typename T> cudaError_t adjoint_fwd_table(sipf_adjoint* a) {
  const sipf_ctx* c = a->c;
  const size_t H3 = (size_t)c->H3(), S = (size_t)c->S();
  FftRun<T> r[3];
  for (int d = 0; d < 3; ++d) {
    r[d] = FftRun<T>{};
    r[d].phi = (T*)a->gbar + d * H3;
    r[d].phi_fixed = 0;
    r[d].in_scale = 1.0;
    r[d].T1 = (cpx<T>*)a->ghat + d * S;
  }
  cudaError_t e = cudaMalloc(&a->fwd_tab, sizeof(r));
  if (e == cudaSuccess) e = cudaMemcpy(a->fwd_tab, r, sizeof(r), cudaMemcpyHostToDevice);
  return e;
}

// Put the context in state (X in id order, alpha, step n): re-bin and deposit.
template <typename T> int load_state(sipf_ctx* c, const T* X, const void* alpha, int64_t n) {
  const size_t P = (size_t)c->p.P;
  for (int d = 0; d < 3; ++d)
    SIPF_CK(cudaMemcpyAsync(c->st[d], X + d * P, P * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
  SIPF_CK(launch_iota(c->st_id, c->p.P, c->stream));
  SIPF_CK(cudaMemcpyAsync(c->alpha, alpha, (size_t)c->S() * 2 * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
  c->n = n;
  return rebin_from_staging<T>(c);
}

template <typename T> int adjoint_forward_impl(sipf_adjoint* a, double* rho_out) {
  sipf_ctx* c = a->c;
  const size_t P = (size_t)c->p.P, S2 = (size_t)c->S() * 2;
  T* ckX = (T*)a->ckX;
  T* ckA = (T*)a->ckA;
  SIPF_CK(cudaEventRecord(a->ev[0], c->stream));
  SIPF_CK(cudaMemsetAsync(c->alpha, 0, S2 * sizeof(T), c->stream));
  SIPF_CK(cudaMemsetAsync(c->dsc, 0, kDscCount * sizeof(double), c->stream));
  c->n = 0;
  int r = upload_aos<T>(c, a->X0.data());
  if (r) return r;
  for (int64_t n = 1; n <= a->N; ++n) {
    if ((n - 1) % a->C == 0) {
      const int64_t k = (n - 1) / a->C;
      T* X = ckX + (size_t)k * 3 * P;
      r = positions_dev_impl<T>(c, X, X + P, X + 2 * P);
      if (r) return r;
      SIPF_CK(cudaMemcpyAsync(ckA + (size_t)k * S2, c->alpha, S2 * sizeof(T), cudaMemcpyDeviceToDevice, c->stream));
    }
    r = step_impl<T>(c, 1);
    if (r) return r;
  }
  T* XN = (T*)a->XN;
  r = positions_dev_impl<T>(c, XN, XN + P, XN + 2 * P);
  if (r) return r;
  SIPF_CK(cudaEventRecord(a->ev[1], c->stream));
  if (rho_out) {
    r = density_host<T>(c, rho_out, 0);
    if (r) return r;
  }
  a->have_forward = true;
  return SIPF_OK;
}

template <typename T>
int adjoint_backward_impl(sipf_adjoint* a, const double* rho_bar, double* grad_chi, double* grad_mu, double* grad_X0) {
  sipf_ctx* c = a->c;
  const sipf_params& p = c->p;
  const int H = p.H, nh = H / 2 + 1;
  const size_t P = (size_t)p.P, H3 = (size_t)c->H3(), S = (size_t)c->S();
  const Geo<T> geo = make_geo<T>(p.L, H);
  const double h3 = pow(p.L / H, 3);
  const T w_inv_h = (T)(p.mass / (double)p.P * H / p.L);
  cudaStream_t s = c->stream;
  SIPF_CK(cudaEventRecord(a->ev[2], s));
  {
    std::vector<T> hb(H3);
    for (size_t i = 0; i < H3; ++i) hb[i] = (T)(rho_bar[i] / h3);
    SIPF_CK(cudaMemcpyAsync(a->phibar, hb.data(), H3 * sizeof(T), cudaMemcpyHostToDevice, s));
    SIPF_CK(cudaStreamSynchronize(s));
  }
  T* XN = (T*)a->XN;
  T* xb = (T*)a->xb;
  SIPF_CK(launch_adj_terminal<T>(XN, XN + P, XN + 2 * P, p.P, (const T*)a->phibar, p.p2g_order, w_inv_h, geo, xb, s));
  a->launches += 1;
  SIPF_CK(cudaMemsetAsync(a->abar, 0, S * 2 * sizeof(T), s));
  SIPF_CK(cudaMemsetAsync(a->phibar, 0, H3 * sizeof(T), s));   // phibar^{N-1} = L^-3 F^-1 (B abar^N) = 0
  SIPF_CK(cudaMemsetAsync(a->phibar4, 0, 4 * H3 * sizeof(T), s));
  SIPF_CK(cudaMemsetAsync(a->acc, 0, 2 * sizeof(double), s));
  const double sn = p.splitting == SIPF_SPLIT_HALF ? sqrt(p.mu * p.dt) : sqrt(2.0 * p.mu * p.dt);
  SpecParams sp = spec_params(c);
  T* segX = (T*)a->segX;
  uint32_t* segI = a->segI;
  T* segG = (T*)a->segG;
  for (int k = a->nck - 1; k >= 0; --k) {
    const int64_t k0 = (int64_t)k * a->C, k1 = std::min<int64_t>(k0 + a->C, a->N);
    int r = load_state<T>(c, (const T*)a->ckX + (size_t)k * 3 * P, (const T*)a->ckA + (size_t)k * 2 * S, k0);
    if (r) return r;
    for (int64_t j = k0; j < k1; ++j) {
      // X^j in the order of the current tile bins, with the particle ids
      T* X = segX + (size_t)(j - k0) * 3 * P;
      SIPF_CK(launch_compact<T>(bin_args<T>(c, c->cur, c->lc, -1, 0), c->max_chunks(), a->cursor, X, X + P, X + 2 * P,
                                segI + (size_t)(j - k0) * P, s));
      a->launches += 1;
      r = step_impl<T>(c, 1);
      if (r) return r;
      // after step j+1 the context's gradient buffer holds g^{j}
      SIPF_CK(cudaMemcpyAsync(segG + (size_t)(j - k0) * 4 * H3, c->grad, 4 * H3 * sizeof(T), cudaMemcpyDeviceToDevice,
                              s));
    }
    for (int64_t n = k1; n > k0; --n) {
      const size_t i = (size_t)(n - 1 - k0);
      AdjArgs<T> aa{};
      aa.x = segX + i * 3 * P;
      aa.y = aa.x + P;
      aa.z = aa.x + 2 * P;
      aa.id = segI + i * P;
      aa.grad4 = segG + i * 4 * H3;
      aa.phibar = (const T*)a->phibar;
      aa.phibar4 = (const T*)a->phibar4;
      aa.xb4 = xb;
      aa.gbar = (T*)a->gbar4;
      aa.acc = a->acc;
      aa.g = geo;
      aa.s_noise = (T)sn;
      aa.chitau = (T)(p.chi * p.dt);
      aa.tau = (T)p.dt;
      aa.w_inv_h = w_inv_h;
      aa.seed = p.seed;
      aa.n = (uint32_t)n;
      aa.P = p.P;
      aa.p2g = p.p2g_order;
      aa.g2p = p.g2p_order;
      aa.split = p.splitting;
      SIPF_CK(launch_adj_step<T>(aa, s));
      SIPF_CK(launch_adj_planes<T>((T*)a->gbar4, (T*)a->gbar, (int64_t)H3, s));
      // ghat = unnormalised DFT of the three cotangent grids
      cpx<T>* gh = (cpx<T>*)a->ghat;
      if (a->fwd_tab) {
        int fk = 0;
        SIPF_CK(launch_field_batch<T>((const FftRun<T>*)a->fwd_tab, 3, H, kFieldForward, s, FieldTune{}, &fk));
        a->launches += fk - 2;
      } else {
        SIPF_CK(launch_rows_r2c<T>(a->gbar, 0, 1.0, false, gh, H, 3 * H * H, nullptr, s));
        SIPF_CK(launch_cols<T>(gh, H, 3 * H, nh, 1, 0, -1, 1.0, s));
      }
      SIPF_CK(launch_cols<T>(gh, H, 1, H * nh, 3, S, -1, 1.0, s));
      // abar^{n-1} = A abar^n + Gop^T gbar;  spec = L^-3 B abar^{n-1}
      cpx<T>* sc = (cpx<T>*)a->spec;
      SIPF_CK(launch_adj_spectral<T>(gh, (cpx<T>*)a->abar, sc, H, sp, s));
      // phibar^{n-2} = F^-1(spec)
      SIPF_CK(launch_cols<T>(sc, H, 1, H * nh, 1, 0, +1, 1.0, s));
      SIPF_CK(launch_cols<T>(sc, H, H, nh, 1, 0, +1, 1.0, s));
      SIPF_CK(launch_rows_c2r<T>(sc, 1, 0, (T*)a->phibar, H, H * H, nullptr, s));
      SIPF_CK(launch_adj_quads<T>((const T*)a->phibar, (T*)a->phibar4, H, s));
      a->launches += 10;
    }
  }
  SIPF_CK(cudaEventRecord(a->ev[3], s));
  double acc[2];
  SIPF_CK(cudaMemcpyAsync(acc, a->acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  std::vector<T> h;
  if (grad_X0) {
    h.resize(4 * P);
    SIPF_CK(cudaMemcpyAsync(h.data(), xb, 4 * P * sizeof(T), cudaMemcpyDeviceToHost, s));
  }
  SIPF_CK(cudaStreamSynchronize(s));
  if (grad_chi) *grad_chi = acc[0];
  if (grad_mu) *grad_mu = acc[1] * sn / (2.0 * p.mu);
  if (grad_X0)
    for (size_t i = 0; i < P; ++i)
      for (int d = 0; d < 3; ++d) grad_X0[3 * i + d] = (double)h[4 * i + d];
  return SIPF_OK;
}

}  // namespace

extern "C" {

int sipf_adjoint_init(const sipf_params* p, const double* X0, int64_t nsteps, int32_t checkpoint_every, void* stream,
                      sipf_adjoint** out) {
  if (!out) return fail(SIPF_EINVAL, "out is NULL");
  *out = nullptr;
  int v = validate(p);
  if (v) return v;
  if (!X0) return fail(SIPF_EINVAL, "X0 is NULL");
  if (nsteps < 1 || nsteps > 0xFFFFFFFFLL) return fail(SIPF_EINVAL, "nsteps (1 <= nsteps < 2^32)");
  if (checkpoint_every < 0) return fail(SIPF_EINVAL, "checkpoint_every (>= 0)");
  if (!(p->mu > 0)) return fail(SIPF_EINVAL, "the adjoint needs mu > 0 (dJ/dmu goes through sqrt(mu tau))");
  sipf_adjoint* a = new sipf_adjoint();
  a->N = nsteps;
  a->C = checkpoint_every > 0 ? checkpoint_every : kAdjCheckpoint;
  if (a->C > nsteps) a->C = (int)nsteps;
  a->nck = (int)((nsteps + a->C - 1) / a->C);
  a->X0.assign(X0, X0 + 3 * p->P);
  int r = sipf_init(p, X0, stream, &a->c);
  if (r) {
    delete a;
    return r;
  }
  sipf_ctx* c = a->c;
  const size_t esz = c->esz, P = (size_t)p->P, H3 = (size_t)c->H3(), S = (size_t)c->S();
  cudaError_t e = cudaMalloc(&a->ckX, (size_t)a->nck * 3 * P * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->ckA, (size_t)a->nck * 2 * S * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->segX, (size_t)a->C * 3 * P * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->segI, (size_t)a->C * P * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&a->cursor, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&a->segG, (size_t)a->C * 4 * H3 * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->XN, 3 * P * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->xb, 4 * P * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->abar, 2 * S * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->spec, 2 * S * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->gbar, 3 * H3 * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->gbar4, 4 * H3 * esz);
  if (e == cudaSuccess) e = cudaMemset(a->gbar4, 0, 4 * H3 * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->ghat, 3 * 2 * S * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->phibar, H3 * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->phibar4, 4 * H3 * esz);
  if (e == cudaSuccess) e = cudaMalloc(&a->acc, 2 * sizeof(double));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&a->ev[i]);
  if (e == cudaSuccess && p->H >= 32)
    e = p->precision == 64 ? adjoint_fwd_table<double>(a) : adjoint_fwd_table<float>(a);
  if (e != cudaSuccess) {
    adjoint_free(a);
    return cuda_fail(e, "sipf_adjoint_init allocation");
  }
  *out = a;
  return SIPF_OK;
}

int sipf_adjoint_forward(sipf_adjoint* a, double chi, double mu, const double* X0, double* rho_out) {
  if (!a) return fail(SIPF_EINVAL, "adjoint is NULL");
  if (!(isfinite(chi) && chi >= 0)) return fail(SIPF_EINVAL, "chi (>= 0)");
  if (!(isfinite(mu) && mu > 0)) return fail(SIPF_EINVAL, "mu (> 0)");
  if (X0) {
    for (int64_t i = 0; i < 3 * a->c->p.P; ++i)
      if (!isfinite(X0[i])) return fail(SIPF_ENONFINITE, "X0 holds a non-finite coordinate");
    a->X0.assign(X0, X0 + 3 * a->c->p.P);
  }
  a->c->p.chi = chi;
  a->c->p.mu = mu;
  a->have_forward = false;
  int r = DISPATCH(a->c, adjoint_forward_impl, a, rho_out);
  if (r) return r;
  return sipf_sync(a->c);
}

int sipf_adjoint_backward(sipf_adjoint* a, const double* rho_bar, double* grad_chi, double* grad_mu,
                          double* grad_X0) {
  if (!a || !rho_bar) return fail(SIPF_EINVAL, "adjoint or rho_bar is NULL");
  if (!a->have_forward) return fail(SIPF_EINVAL, "sipf_adjoint_backward needs a preceding sipf_adjoint_forward");
  int r = DISPATCH(a->c, adjoint_backward_impl, a, rho_bar, grad_chi, grad_mu, grad_X0);
  if (r) return r;
  return sipf_sync(a->c);
}

int sipf_adjoint_timing(const sipf_adjoint* a, double* forward_ms, double* backward_ms) {
  if (!a) return fail(SIPF_EINVAL, "adjoint is NULL");
  float f = 0.f, b = 0.f;
  if (forward_ms) {
    SIPF_CK(cudaEventSynchronize(a->ev[1]));
    SIPF_CK(cudaEventElapsedTime(&f, a->ev[0], a->ev[1]));
    *forward_ms = f;
  }
  if (backward_ms) {
    SIPF_CK(cudaEventSynchronize(a->ev[3]));
    SIPF_CK(cudaEventElapsedTime(&b, a->ev[2], a->ev[3]));
    *backward_ms = b;
  }
  return SIPF_OK;
}

int sipf_measure_fp64_fma(void* stream, double* gflops) {
  if (!gflops) return fail(SIPF_EINVAL, "gflops is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  SIPF_CK(cudaGetDevice(&dev));
  SIPF_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* sink = nullptr;
  SIPF_CK(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * 8, iters = 1 << 14;
  if (e == cudaSuccess) e = launch_fp64_fma(blocks, 64, sink, s);   // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) e = launch_fp64_fma(blocks, iters, sink, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "sipf_measure_fp64_fma");
  *gflops = 2.0 * blocks * 256.0 * 8.0 * iters / (ms * 1e-3) / 1e9;
  return SIPF_OK;
}

int64_t sipf_adjoint_kernel_launches(const sipf_adjoint* a) { return a ? a->c->launches + a->launches : -1; }

void sipf_adjoint_destroy(sipf_adjoint* a) { adjoint_free(a); }

}  // extern "C"
