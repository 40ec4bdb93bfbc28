// C ABI of the MFA library: layout builder, device tables, the launch
// sequences of encode (setup + iteration 0), the Schwarz loop, decode and
// residual.  See include/mfa.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "mfa_internal.cuh"

using namespace mfa;

// ---------------------------------------------------------------------------
// handle and model
// ---------------------------------------------------------------------------

namespace {
struct PlanCache;
// host data of a fused 3-D encode is copied in this many z-slabs, the
// projection units of each slab launched as it lands
constexpr int kSlabs = 16;
}  // namespace

struct mfa_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaMemPool_t pool = nullptr;
  int* d_status = nullptr;
  unsigned long long* d_metrics = nullptr;  // [4]
  double* d_partials = nullptr;             // [4 * kResidualBlocks]
  double* d_result = nullptr;               // [4]
  double* h_pinned = nullptr;               // [16] readback
  char* h_stage = nullptr;                  // pinned staging of layout tables (grown as needed)
  size_t h_stage_cap = 0;
  cudaEvent_t stage_done = nullptr;         // the last upload from h_stage has been read
  char* h_stage32 = nullptr;                // pinned staging of FP32 batch tables (grown as needed)
  size_t h_stage32_cap = 0;
  cudaEvent_t stage32_done = nullptr;       // the last upload from h_stage32 has been read
  cudaStream_t copy_stream = nullptr;       // host data copied slab by slab beside the projection
  std::vector<cudaEvent_t> slab_ev;         // slab landed (copy stream) / buffers allocated (handle stream)
  void* rb = nullptr;                       // staging of asynchronous control-point reads
  size_t rb_size = 0;
  cudaEvent_t rb_ready = nullptr;           // rb written (handle stream)
  cudaEvent_t rb_done = nullptr;            // rb copied out (copy stream)
  PlanCache* plan = nullptr;                // host products of the most recent single-model layout
  void (*plan_free)(PlanCache*) = nullptr;  // its deleter (set with it)
  bool plan_valid = false;                  // plan matches the image in h_stage
  void* ws = nullptr;                       // growable scratch
  size_t ws_size = 0;
  int live_models = 0;
  // tracing: per-class CUDA-event timing and launch counts
  bool trace_on = false;
  double trace_ms[MFA_TRACE_CLASSES] = {};
  long long trace_n[MFA_TRACE_CLASSES] = {};
  std::vector<cudaEvent_t> ev;               // event pool, used in pairs
  std::vector<std::pair<int, int>> pending;  // (class, first event index)
  int ev_next = 0;
};

struct mfa_model {
  mfa_handle* h = nullptr;
  const void* q_staged = nullptr;  // device copy of host data given to mfa_encode (inside `big`)
  int q_staged_dtype = MFA_F32;
  bool plain = false;              // per-subdomain comparator form (mfa_encode_plain)
  bool batch = false;              // one (dimension, degree) group of a batch of independent fits
  bool has_state = false;          // B_L and the subdomain copies are valid (the Schwarz iteration can run)
  int overlap[3] = {0, 0, 0};      // delta per axis, as given
  int update = UPDATE_AVERAGE;     // rule of the global update from the owned copies
  long long maxDec[3] = {0, 0, 0}; // batch: largest decode-stage output per axis
  long long decS1 = 0, decS2 = 0;  // batch: decode stage scratch sizes (elements)
  TileMap tm_proj[3], tm_solve[3], tm_dec[3];  // batch: compact launches over the uneven instances
  void* tiles = nullptr;                       // device storage of the tile maps
  const int* res_first = nullptr;              // batch: first last-axis decode tile of every instance [nsub + 1]
  const int* res_id = nullptr;                 // batch: batch index of every instance of the group [nsub]
  const int* order = nullptr;                  // batch: instances largest first (fused projection CTA order)
  std::vector<AxisOp> hops;                    // batch: host copy of the operand tables (tile maps are rebuilt from it)
  std::vector<int> hmem;                       // batch: batch index of every instance of the group
  int tile_c = 0, tile_s = 0, tile_e = 0;      // batch: block sizes of the current tile maps
  float tune_ms[MFA_TUNE_CANDIDATES] = {};     // batch: this group's timed candidates (-1: not run)
  float tune_best = 0.f;                       // batch: time of the chosen candidate
  const void* q_src = nullptr;     // plain form: the device data it re-reads every iteration
  int q_src_dtype = MFA_F32;
  int prec = MFA_PREC_FP64;
  int knots = MFA_KNOTS_FLOATING;  // knots at the interfaces, as given in the layout
  int dim = 1;
  int degree = 1;
  double last_rms = -1.0;          // decoded RMS of the current iterate, when the stall test has computed it
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  AxisHost axh[3];
  LayoutDev L{};
  int nsub = 1;
  long long sizeL = 0, sizeS1 = 0, sizeS2 = 0;
  int maxL = 0, maxU = 0, maxS1 = 0, maxS2 = 0;
  int maxm[3] = {0, 0, 0}, maxnL[3] = {0, 0, 0}, maxnU[3] = {0, 0, 0};  // largest window points / L / U per axis
  int maxOut[3] = {0, 0, 0};      // projection stage output sizes
  int maxApply[3] = {0, 0, 0};    // band-apply output sizes
  int maxFibL[3] = {0, 0, 0};     // fibres per solve, L boxes
  int maxFibU[3] = {0, 0, 0};
  void* arena = nullptr;          // device tables
  void* big = nullptr;            // B_L, X, P, Pprev, S1, S2
  // device pointers inside the arena
  long long *offL = nullptr, *offS1 = nullptr, *offS2 = nullptr;
  AxisOp* ops = nullptr;  // [kOpKinds][nsub]
  // big buffers
  void *BL = nullptr, *X = nullptr, *P = nullptr, *Pprev = nullptr, *S1 = nullptr, *S2 = nullptr;
  float* part = nullptr;  // per-block metric partials of the float-float average
  int zsplit = 1;         // fused projection: units per window along z
  const int2* units = nullptr;   // its (subdomain, unit) pairs by the slab their last plane lands in
  std::vector<int> slab_units;   // units of slabs < t: slab_units[t] (kSlabs + 1 entries)
  long long slab_planes = 0;     // z-planes per slab of host data
  ff* zpart = nullptr;    // its partial sums of shared z-control points
  unsigned* zctr = nullptr;
  bool use_fused = true;     // fused 3-D kernels where they cover the layout
  bool x_inplace_ok = true;  // every x-window has >= 2 points per span (in-place stage-1 output)
  int iters = 0;
  int grow_streak = 0;
  double last_dP = 0.0;
  double last_jump = 0.0;
};

namespace mfa {
int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) return 1;
  if (dev >= 0 && dev < 64) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}
}  // namespace mfa

namespace {

// op table rows
enum OpKind { OP_PROJ0 = 0, OP_PROJ1, OP_PROJ2, OP_SOLVEL0, OP_SOLVEL1, OP_SOLVEL2, OP_APPLY0, OP_APPLY1, OP_APPLY2,
              OP_SOLVEU0, OP_SOLVEU1, OP_SOLVEU2, OP_DEC0, OP_DEC1, OP_DEC2, kOpKinds };

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Highest float of a staged row written by the fused projection's stage-1
// output of control points 0..c (16-byte groups of two control points).
inline long long stage1_reach(long long c) { return (c & 1) ? 2 * c + 1 : 2 * c + 2; }

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MFA_OK;
  if (e == cudaErrorMemoryAllocation) return MFA_ERR_OOM;
  return MFA_ERR_CUDA;
}

int pool_alloc(mfa_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? MFA_ERR_OOM : MFA_ERR_CUDA;
  }
  return MFA_OK;
}

void pool_free(mfa_handle* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

int ensure_ws(mfa_handle* h, size_t bytes) {
  if (h->ws_size >= bytes) return MFA_OK;
  pool_free(h, h->ws);
  h->ws = nullptr;
  h->ws_size = 0;
  int rc = pool_alloc(h, &h->ws, bytes);
  if (rc == MFA_OK) h->ws_size = bytes;
  return rc;
}

// ---------------------------------------------------------------------------
// tracing
// ---------------------------------------------------------------------------

enum TraceClass {
  TR_SETUP = 0,        // basis tables, Gram bands, Cholesky factors
  TR_PROJECT_DATA,     // first projection stage: reads the data
  TR_PROJECT_REDUCED,  // later projection stages on reduced arrays
  TR_SOLVE_L,          // iteration-0 banded solves
  TR_AVERAGE,          // 1/n_s averaging + metrics
  TR_FRAME_GATHER,     // Schwarz exchange
  TR_BAND_APPLY,       // coupling product G P_F
  TR_RHS_FINALIZE,     // B_U - G P_F
  TR_SOLVE_U,          // owned-box banded solves
  TR_DECODE_STAGE,     // intermediate decode stages
  TR_RESIDUAL,         // last decode stage fused with the residual + reduction
  TR_DECODE_OUT,       // last decode stage writing the output grid
  TR_DECODE_POINTS,    // scattered decode
  TR_MISC,             // casts
  TR_REDUCE,           // final fixed-order reduction of residual partials
  TR_REFINE_DATA       // refinement projection of r = q - N P (MFA_PREC_FP32 batches)
};

const char* kTraceNames[MFA_TRACE_CLASSES] = {
    "setup_basis_gram_chol", "project_data", "project_reduced", "solve_iter0", "average", "frame_gather",
    "band_apply", "rhs_finalize", "solve_owned", "decode_stage", "residual", "decode_out", "decode_points",
    "cast", "reduce", "refine_data"};

void trace_flush(mfa_handle* h) {
  if (h->pending.empty()) {
    h->ev_next = 0;
    return;
  }
  cudaEventSynchronize(h->ev[h->pending.back().second + 1]);
  cudaStreamSynchronize(h->stream);  // events recorded on a batch's side streams are joined into it
  for (auto& pr : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[pr.second], h->ev[pr.second + 1]) == cudaSuccess)
      h->trace_ms[pr.first] += ms;
  }
  cudaGetLastError();
  h->pending.clear();
  h->ev_next = 0;
}

int trace_begin(mfa_handle* h) {
  if (!h->trace_on) return -1;
  if (h->ev_next + 2 > (int)h->ev.size()) trace_flush(h);
  const int i = h->ev_next;
  cudaEventRecord(h->ev[i], h->stream);
  return i;
}

void trace_end(mfa_handle* h, int cls, int i, int nlaunch = 1) {
  h->trace_n[cls] += nlaunch;
  if (i < 0) return;
  cudaEventRecord(h->ev[i + 1], h->stream);
  h->pending.push_back({cls, i});
  h->ev_next = i + 2;
}

#define TRACED(h, cls, stmt)        \
  do {                              \
    const int _ti = trace_begin(h); \
    stmt;                           \
    trace_end(h, cls, _ti);         \
  } while (0)

// same, for a call that launches `n` kernels
#define TRACED_N(h, cls, n, stmt)     \
  do {                                \
    const int _ti = trace_begin(h);   \
    stmt;                             \
    trace_end(h, cls, _ti, (n));      \
  } while (0)

// ---------------------------------------------------------------------------
// layout builder (Sec. 2.2): cores, windows, data ranges, U/L sets, owners
// ---------------------------------------------------------------------------

// Does control point g have a nonzero basis value at data point k?  Exact in
// integers with the knot positions t_i = kn[i] / gspans: N_g is positive on
// the open interval (t_g, t_{g+p+1}), at its left end when the knot there has
// multiplicity p+1 (a clamped start), and the last function at u = 1.
bool in_support(const AxisHost& ax, long long k, int g) {
  if (ax.M == 1) return true;
  const long long x = k * ax.gspans, M1 = ax.M - 1;
  const long long lo = ax.knots[g], hi = ax.knots[g + ax.p + 1];
  if (lo * M1 < x && x < hi * M1) return true;
  if (x == lo * M1 && ax.knots[g + ax.p] == lo && lo < hi) return true;
  return g == ax.n - 1 && k == ax.M - 1;
}

// Schoenberg-Whitney condition for the window's collocation matrix: a
// strictly increasing assignment of data points to the L control points with
// nonzero basis value.  Greedy in control-point order.
bool schoenberg_whitney(const AxisHost& ax, const AxisSub& sb) {
  long long next = sb.k0;
  for (int l = 0; l < sb.nL; ++l) {
    const int g = sb.l0 + l;
    bool found = false;
    for (long long k = next; k < sb.k0 + sb.m; ++k) {
      if (in_support(ax, k, g)) {
        next = k + 1;
        found = true;
        break;
      }
    }
    if (!found) return false;
  }
  return true;
}

// Layout of one axis (Sec. 2.2).  Floating knots: single interior knots,
// span j carries control points j .. j+p.  Clamped interfaces (Sec. 2.2 /
// Sec. 3.1.1 variant): every interface breakpoint is repeated p times, so the
// first control point of span j is j + (p-1) * (number of interfaces at or
// before j), each core carries its own clamped uniform knot vector, and
// neighbours share the single control point at their interface.  Spans are
// numbered by their first control point throughout (`nspans` then counts the
// span numbers, `gspans` the grid's knot spans).
int build_axis(AxisHost& ax, long long M, int nspans, int p, int nsub, const int32_t* core, int delta,
               int knots = MFA_KNOTS_FLOATING) {
  if (M < 1 || M > (1LL << 30)) return MFA_ERR_ARG;
  if (knots != MFA_KNOTS_FLOATING && knots != MFA_KNOTS_CLAMPED) return MFA_ERR_ARG;
  if (nspans < 1 || nsub < 1 || nsub > nspans || delta < 0) return MFA_ERR_LAYOUT;
  // clamping changes nothing for p <= 1 or a single core
  const bool clamped = knots == MFA_KNOTS_CLAMPED && p > 1 && nsub > 1;
  ax.M = (int)M;
  ax.gspans = nspans;
  ax.p = p;
  ax.S = nsub;
  ax.kmode = clamped ? KMODE_CLAMPED : KMODE_FLOATING;
  std::vector<int> cs(nsub);
  if (core) {
    long long tot = 0;
    for (int s = 0; s < nsub; ++s) {
      cs[s] = core[s];
      tot += core[s];
    }
    if (tot != nspans) return MFA_ERR_LAYOUT;
  } else {
    for (int s = 0; s < nsub; ++s) cs[s] = nspans / nsub + (s < nspans % nsub ? 1 : 0);
  }
  // cores between interfaces need >= p spans; a single subdomain has none
  std::vector<int> piece_of_span(nspans, 0), core_start(nsub + 1, 0);
  for (int s = 0; s < nsub; ++s) {
    if (nsub > 1 && cs[s] < std::max(p, 1)) return MFA_ERR_LAYOUT;
    core_start[s + 1] = core_start[s] + cs[s];
    for (int j = core_start[s]; j < core_start[s + 1]; ++j) piece_of_span[j] = s;
  }
  // first control point of span j; knot positions (multiplicity p at clamped interfaces)
  auto first_cp = [&](int j) { return clamped ? j + (p - 1) * piece_of_span[j] : j; };
  ax.nspans = first_cp(nspans - 1) + 1;
  ax.n = ax.nspans + p;
  ax.knots.assign(p + 1, 0);
  for (int i = 1; i < nspans; ++i) {
    const bool iface = clamped && piece_of_span[i] != piece_of_span[i - 1];
    for (int r = 0; r < (iface ? p : 1); ++r) ax.knots.push_back(i);
  }
  for (int r = 0; r <= p; ++r) ax.knots.push_back(nspans);
  if ((int)ax.knots.size() != ax.n + p + 1) return MFA_ERR_LAYOUT;
  ax.subs.clear();
  int bandL = 0, bandU = 0;
  for (int s = 0; s < nsub; ++s) {
    AxisSub sb{};
    sb.a = core_start[s];
    sb.b = core_start[s + 1];
    sb.w0 = std::max(sb.a - delta, 0);
    sb.w1 = std::min(sb.b + delta, nspans);
    // closed window [w0/nspans, w1/nspans]: w0 (M-1) <= k nspans <= w1 (M-1)
    if (M == 1) {
      sb.k0 = 0;
      sb.m = 1;
    } else {
      const long long k0 = (sb.w0 * (M - 1) + nspans - 1) / nspans;  // ceil
      const long long k1 = (sb.w1 * (M - 1)) / nspans;                 // floor
      if (k1 < k0) return MFA_ERR_LAYOUT;
      sb.k0 = (int)k0;
      sb.m = (int)(k1 - k0 + 1);
    }
    sb.l0 = first_cp(sb.w0);
    sb.nL = first_cp(sb.w1 - 1) + p + 1 - sb.l0;
    sb.oU = first_cp(sb.a) - sb.l0;
    sb.nU = first_cp(sb.b - 1) + p + 1 - first_cp(sb.a);
    sb.bandL = bandL;
    sb.bandU = bandU;
    bandL += sb.nL;
    bandU += sb.nU;
    if (!schoenberg_whitney(ax, sb)) return MFA_ERR_LAYOUT;
    ax.subs.push_back(sb);
  }
  ax.bandL_rows = bandL;
  ax.bandU_rows = bandU;
  // owners of every global control point (1 or 2 per axis since cores >= p)
  ax.own_first.assign(ax.n, -1);
  ax.own_count.assign(ax.n, 0);
  for (int s = 0; s < nsub; ++s) {
    const AxisSub& sb = ax.subs[s];
    for (int g = sb.l0 + sb.oU; g < sb.l0 + sb.oU + sb.nU; ++g) {
      if (ax.own_first[g] < 0) ax.own_first[g] = s;
      ax.own_count[g]++;
    }
  }
  for (int g = 0; g < ax.n; ++g)
    if (ax.own_count[g] < 1 || ax.own_count[g] > 2) return MFA_ERR_LAYOUT;
  ax.own_tab.assign(ax.n, int4{0, 0, -1, 0});
  for (int g = 0; g < ax.n; ++g) {
    const int f = ax.own_first[g];
    ax.own_tab[g].x = f;
    ax.own_tab[g].y = g - ax.subs[f].l0;
    if (ax.own_count[g] == 2) {
      ax.own_tab[g].z = f + 1;
      ax.own_tab[g].w = g - ax.subs[f + 1].l0;
    }
  }
  ax.nL_tab.resize(nsub);
  for (int s = 0; s < nsub; ++s) ax.nL_tab[s] = ax.subs[s].nL;
  // control points owned by one piece alone: contiguous, since the U boxes of
  // neighbouring pieces overlap only at their ends
  ax.one_rng.assign(nsub, int2{0, 0});
  for (int s = 0; s < nsub; ++s) {
    int lo = -1, hi = -1;
    const AxisSub& sb = ax.subs[s];
    for (int g = sb.l0 + sb.oU; g < sb.l0 + sb.oU + sb.nU; ++g)
      if (ax.own_count[g] == 1) {
        if (lo < 0) lo = g;
        hi = g + 1;
      }
    if (lo < 0) continue;
    for (int g = lo; g < hi; ++g)
      if (ax.own_count[g] != 1 || ax.own_first[g] != s) return MFA_ERR_LAYOUT;
    ax.one_rng[s] = int2{lo, hi};
  }
  // owner-takes update: the owner of control point g is the subdomain whose
  // core holds its Greville abscissa xi_g = (t_{g+1} + ... + t_{g+p}) / p;
  // with t_i = kn_i / nspans, xi_g * nspans * p = sum of the kn_i, exact
  ax.own_pick.assign(ax.n, 0);
  for (int g = 0; g < ax.n; ++g) {
    long long S = 0, den = p;
    if (p > 0) {
      for (int i = g + 1; i <= g + p; ++i) S += ax.knots[i];
    } else {
      S = ax.knots[g] + ax.knots[g + 1];
      den = 2;
    }
    int owner = -1;
    for (int s = 0; s < nsub && owner < 0; ++s) {
      const AxisSub& sb = ax.subs[s];
      if (sb.a * den <= S && (S < sb.b * den || (s == nsub - 1 && S <= sb.b * den))) owner = s;
    }
    if (owner == ax.own_first[g])
      ax.own_pick[g] = 0;
    else if (ax.own_count[g] == 2 && owner == ax.own_first[g] + 1)
      ax.own_pick[g] = 1;
    else
      return MFA_ERR_LAYOUT;  // the Greville owner always owns the point; guard against a broken layout
  }
  // first data point of every span number (span of point k = floor(k nspans / (M-1)), capped, then numbered
  // by its first control point; unused numbers start where the next span does)
  ax.span_start.assign(ax.nspans + 1, (int)M);
  int j = 0;
  for (long long k = 0; k < M; ++k) {
    long long sk = (M == 1) ? 0 : (k * nspans) / (M - 1);
    if (sk > nspans - 1) sk = nspans - 1;
    const int v = first_cp((int)sk);
    while (j <= v) ax.span_start[j++] = (int)k;
  }
  return MFA_OK;
}

}  // namespace

namespace {

// Byte sizes of the element type the model computes in.
inline size_t elem_size(int prec) { return prec == MFA_PREC_FP64 ? sizeof(double) : sizeof(ff); }
// control points held in FP64 (MFA_PREC_FP64); float-float for
// MFA_PREC_MIXED and for MFA_PREC_FP32 batches (their banded solves run in
// float-float on the FP32 pipes: this GPU's FP64 rate is a small fraction)
inline bool f64_store(int prec) { return prec == MFA_PREC_FP64; }

View make_view(long long off, int n0, int n1, int n2, long long s0, long long s1, long long s2) {
  View v;
  v.off = off;
  v.n[0] = n0;
  v.n[1] = n1;
  v.n[2] = n2;
  v.st[0] = s0;
  v.st[1] = s1;
  v.st[2] = s2;
  return v;
}

View contiguous(long long off, int n0, int n1, int n2) {
  return make_view(off, n0, n1, n2, 1, n0, (long long)n0 * n1);
}

// Build every per-subdomain op table and the buffer offsets of a model.
// Buffers per subdomain s: B_L and X are L-shaped (nL0 x nL1 x nL2) at offL[s];
// S1 holds the first projection stage (nL0 x m1 x m2) and later the band-apply
// ping buffer; S2 holds the second stage (nL0 x nL1 x m2) and the pong buffer.
void build_ops(mfa_model* md, std::vector<AxisOp>& ops, std::vector<long long>& offL, std::vector<long long>& offS1,
               std::vector<long long>& offS2) {
  const int S0 = md->axh[0].S, S1 = md->axh[1].S, S2 = md->axh[2].S;
  const int ns = S0 * S1 * S2;
  ops.assign((size_t)kOpKinds * ns, AxisOp{});
  offL.assign(ns, 0);
  offS1.assign(ns, 0);
  offS2.assign(ns, 0);
  long long aL = 0, a1 = 0, a2 = 0;
  const long long M0 = md->axh[0].M, M1 = md->axh[1].M;
  for (int s = 0; s < ns; ++s) {
    const int sa[3] = {s % S0, (s / S0) % S1, s / (S0 * S1)};
    const AxisSub b[3] = {md->axh[0].subs[sa[0]], md->axh[1].subs[sa[1]], md->axh[2].subs[sa[2]]};
    const int nL[3] = {b[0].nL, b[1].nL, b[2].nL}, nU[3] = {b[0].nU, b[1].nU, b[2].nU};
    const int m[3] = {b[0].m, b[1].m, b[2].m};
    const long long szL = (long long)nL[0] * nL[1] * nL[2];
    const long long sz1 = std::max((long long)nL[0] * m[1] * m[2], szL);
    const long long sz2 = std::max((long long)nL[0] * nL[1] * m[2], szL);
    offL[s] = aL;
    offS1[s] = a1;
    offS2[s] = a2;
    aL += szL;
    a1 += sz1;
    a2 += sz2;
    md->maxL = std::max<long long>(md->maxL, szL);
    for (int a = 0; a < 3; ++a) {
      md->maxm[a] = std::max(md->maxm[a], m[a]);
      md->maxnL[a] = std::max(md->maxnL[a], nL[a]);
      md->maxnU[a] = std::max(md->maxnU[a], nU[a]);
    }
    md->maxU = std::max(md->maxU, nU[0] * nU[1] * nU[2]);
    auto at = [&](int kind) -> AxisOp& { return ops[(size_t)kind * ns + s]; };
    // projection stages: Q window -> S1 -> S2 -> B_L, skipping padded axes
    {
      const int d = md->dim;
      View in = make_view((long long)b[0].k0 + M0 * ((long long)b[1].k0 + M1 * b[2].k0), m[0], m[1], m[2], 1, M0,
                          M0 * M1);
      int cur[3] = {m[0], m[1], m[2]};
      for (int a = 0; a < d; ++a) {
        cur[a] = nL[a];
        const long long off = (a == d - 1) ? offL[s] : (a == 0 ? offS1[s] : offS2[s]);
        View out = contiguous(off, cur[0], cur[1], cur[2]);
        AxisOp& op = at(OP_PROJ0 + a);
        op.in = in;
        op.out = out;
        op.k0 = b[a].k0;
        op.kend = b[a].k0 + b[a].m;
        op.c0 = b[a].l0;
        op.sa = sa[a];
        md->maxOut[a] = std::max<long long>(md->maxOut[a], (long long)cur[0] * cur[1] * cur[2]);
        in = out;
      }
    }
    // iteration-0 solves over the L box of X, and U-box solves of later iterations
    for (int a = 0; a < 3; ++a) {
      AxisOp& opL = at(OP_SOLVEL0 + a);
      opL.out = contiguous(offL[s], nL[0], nL[1], nL[2]);
      opL.sa = sa[a];
      AxisOp& opU = at(OP_SOLVEU0 + a);
      opU.out = make_view(offL[s] + b[0].oU + (long long)nL[0] * (b[1].oU + (long long)nL[1] * b[2].oU), nU[0], nU[1],
                          nU[2], 1, nL[0], (long long)nL[0] * nL[1]);
      opU.sa = sa[a];
      const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      md->maxFibL[a] = std::max(md->maxFibL[a], nL[o1] * nL[o2]);
      md->maxFibU[a] = std::max(md->maxFibU[a], nU[o1] * nU[o2]);
    }
    // band applies: Pt (L box, in S2) -> S1 -> S2 -> S1 (ping-pong), rows restricted to U
    {
      int cur[3] = {nL[0], nL[1], nL[2]};
      View in = contiguous(offS2[s], cur[0], cur[1], cur[2]);
      for (int a = 0; a < md->dim; ++a) {
        cur[a] = nU[a];
        const long long off = (a % 2 == 0) ? offS1[s] : offS2[s];
        View out = contiguous(off, cur[0], cur[1], cur[2]);
        AxisOp& op = at(OP_APPLY0 + a);
        op.in = in;
        op.out = out;
        op.sa = sa[a];
        op.oU = b[a].oU;
        md->maxApply[a] = std::max<long long>(md->maxApply[a], (long long)cur[0] * cur[1] * cur[2]);
        in = out;
      }
    }
  }
  md->sizeL = aL;
  md->sizeS1 = a1;
  md->sizeS2 = a2;
  // global decode stages (one op each): P (n0 x n1 x n2) -> ... -> grid (M0 x M1 x M2)
  {
    int cur[3] = {md->axh[0].n, md->axh[1].n, md->axh[2].n};
    long long off = 0;
    View in = contiguous(0, cur[0], cur[1], cur[2]);
    for (int a = 0; a < md->dim; ++a) {
      cur[a] = md->axh[a].M;
      View out = contiguous(off, cur[0], cur[1], cur[2]);
      AxisOp& op = ops[(size_t)(OP_DEC0 + a) * ns];
      op.in = in;
      op.out = out;
      op.k0 = 0;
      op.kend = md->axh[a].M;
      op.c0 = 0;
      op.sa = 0;
      in = out;
    }
  }
}

struct Arena {
  size_t used = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t off = used;
    used = align256(used + count * sizeof(T));
    return off;
  }
};

template <typename T>
T* at_off(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// Launch the projection N^T Q (all subdomains) and iteration 0.
// Projection B_L of every window, one subdomain per launch and axis (the
// per-subdomain comparator form; the data are read again on every call).
template <typename T, typename TQ>
void plain_project(mfa_model* md, const TQ* q) {
  mfa_handle* h = md->h;
  const LayoutDev& L = md->L;
  const int ns = md->nsub;
  T* BL = (T*)md->BL;
  T* S1 = (T*)md->S1;
  T* S2 = (T*)md->S2;
  auto opsk = [&](int kind) { return md->ops + (size_t)kind * ns; };
  for (int sd = 0; sd < ns; ++sd)
    for (int a = 0; a < md->dim; ++a) {
      T* out = (a == md->dim - 1) ? BL : (a == 0 ? S1 : S2);
      if (a == 0)
        TRACED(h, TR_PROJECT_DATA,
               (launch_contract<T, TQ>(L, 0, opsk(OP_PROJ0) + sd, 1, md->maxOut[0], q, out, h->d_status, h->stream)));
      else
        TRACED(h, TR_PROJECT_REDUCED,
               (launch_contract<T, T>(L, a, opsk(OP_PROJ0 + a) + sd, 1, md->maxOut[a], a == 1 ? S1 : S2, out, nullptr,
                                      h->stream)));
    }
}

// Host data copied slab by slab on the handle's copy stream while the fused
// projection runs (encode from host data): source, device staging buffer, the
// bytes of one z-plane and the number of planes.
struct StagedCopy {
  const void* host;
  void* dev;
  size_t plane_bytes;
  long long planes;
};

// Copy slabs [t0, t1) of the host data on the copy stream, each followed by
// its event.
cudaError_t copy_slabs(mfa_model* md, const StagedCopy& sc, int t0, int t1) {
  mfa_handle* h = md->h;
  cudaError_t e = cudaSuccess;
  for (int t = t0; t < t1 && e == cudaSuccess; ++t) {
    const long long z0 = std::min<long long>((long long)t * md->slab_planes, sc.planes);
    const long long z1 = std::min<long long>(z0 + md->slab_planes, sc.planes);
    if (z1 > z0)
      e = cudaMemcpyAsync((char*)sc.dev + z0 * sc.plane_bytes, (const char*)sc.host + z0 * sc.plane_bytes,
                          (size_t)(z1 - z0) * sc.plane_bytes, cudaMemcpyHostToDevice, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->slab_ev[t], h->copy_stream);
  }
  return e;
}

template <typename T, typename TQ>
void run_encode(mfa_model* md, const TQ* q, const StagedCopy* sc = nullptr) {
  mfa_handle* h = md->h;
  const LayoutDev& L = md->L;
  const int ns = md->nsub;
  T* BL = (T*)md->BL;
  T* X = (T*)md->X;
  T* S1 = (T*)md->S1;
  T* S2 = (T*)md->S2;
  auto opsk = [&](int kind) { return md->ops + (size_t)kind * ns; };
  // projection: the fused 3-D kernel when it covers the layout, else one
  // launch per axis where stage a reads the previous stage (the data for a = 0)
  bool fused = false;
  int slabs_done = 0;  // host data: slabs already copied (all of them once the projection has its data)
  // the fused projection stages FP32 data; FP64 data take the per-axis
  // kernels, which carry them exactly as float-float
  constexpr bool kFusedData = std::is_same<T, ff>::value && std::is_same<TQ, float>::value;
  if constexpr (kFusedData) {
    if (md->dim == 3 && md->use_fused && sc && md->units) {
      // the units of slab t wait for slabs 0..t only, so the projection runs
      // under the rest of the copy
      fused = true;
      for (int t = 0; t < kSlabs && fused; ++t) {
        copy_slabs(md, *sc, t, t + 1);
        slabs_done = t + 1;
        cudaStreamWaitEvent(h->stream, h->slab_ev[t], 0);
        TRACED(h, TR_PROJECT_DATA,
               fused = launch_project3d_ff<TQ>(L, md->offL, md->maxm[0], md->maxm[1], md->maxm[2], md->maxnL[0],
                                                md->maxnL[1], md->x_inplace_ok, q, BL, h->d_status, h->stream,
                                                nullptr, nullptr, md->zsplit, md->zpart, md->zctr,
                                                md->units + md->slab_units[t], md->slab_units[t + 1] - md->slab_units[t],
                                                t == 0));
      }
    }
  }
  if (sc && slabs_done < kSlabs) {
    // every other path reads the whole grid: copy the rest and wait for it
    copy_slabs(md, *sc, slabs_done, kSlabs);
    cudaStreamWaitEvent(h->stream, h->slab_ev[kSlabs - 1], 0);
  }
  if constexpr (kFusedData) {
    if (md->dim == 3 && md->use_fused && !fused) {
      TRACED(h, TR_PROJECT_DATA,
             fused = launch_project3d_ff<TQ>(L, md->offL, md->maxm[0], md->maxm[1], md->maxm[2], md->maxnL[0], md->maxnL[1],
                                              md->x_inplace_ok, q, BL, h->d_status, h->stream,
                                              md->batch ? md->ops + (size_t)OP_PROJ0 * ns : nullptr,
                                              md->batch ? md->order : nullptr, md->zsplit, md->zpart, md->zctr));
    }
  }
  if (md->plain) {
    plain_project<T, TQ>(md, q);
    fused = true;
  }
  for (int a = 0; a < md->dim && !fused; ++a) {
    T* out = (a == md->dim - 1) ? BL : (a == 0 ? S1 : S2);
    if (a == 0)
      TRACED(h, TR_PROJECT_DATA,
             (launch_contract<T, TQ>(L, 0, opsk(OP_PROJ0), ns, md->maxOut[0], q, out, h->d_status, h->stream,
                                     md->batch ? &md->tm_proj[0] : nullptr)));
    else
      TRACED(h, TR_PROJECT_REDUCED,
             (launch_contract<T, T>(L, a, opsk(OP_PROJ0 + a), ns, md->maxOut[a], a == 1 ? S1 : S2, out, nullptr,
                                    h->stream, md->batch ? &md->tm_proj[a] : nullptr)));
  }
  // iteration 0: unconstrained local solves on the L boxes
  int it0 = 0;
  if constexpr (std::is_same<T, ff>::value) {
    if (md->dim == 3 && md->use_fused) {
      const int _ti = trace_begin(h);
      it0 = launch_iter0_3d_ff(L, md->offL, md->maxnL, BL, X, h->stream);
      trace_end(h, TR_SOLVE_L, _ti, it0);
    }
  }
  if (!it0 && X != BL) cudaMemcpyAsync(X, BL, md->sizeL * sizeof(T), cudaMemcpyDeviceToDevice, h->stream);
  for (int a = 0; a < md->dim && !it0; ++a) {
    if (md->plain) {
      for (int sd = 0; sd < ns; ++sd)
        TRACED(h, TR_SOLVE_L,
               launch_band_solve<T>(L, a, false, opsk(OP_SOLVEL0 + a) + sd, 1, md->maxFibL[a], X, h->stream));
    } else {
      TRACED(h, TR_SOLVE_L, launch_band_solve<T>(L, a, false, opsk(OP_SOLVEL0 + a), ns, md->maxFibL[a], X, h->stream,
                                                 md->batch ? &md->tm_solve[a] : nullptr));
    }
  }
  if (md->batch) return;  // one subdomain per instance: the solution is X itself
  cudaMemsetAsync(h->d_metrics, 0, 4 * sizeof(unsigned long long), h->stream);
  if constexpr (std::is_same<T, ff>::value) {
    if (md->use_fused) {
      TRACED_N(h, TR_AVERAGE, 1,
               launch_average_ff(L, md->offL, X, (ff*)md->P, nullptr, md->part, h->d_metrics, h->stream,
                                 md->update));
      return;
    }
  }
  TRACED(h, TR_AVERAGE, launch_average<T>(L, md->offL, X, (T*)md->P, nullptr, h->d_metrics, h->stream, md->update));
}

// One Schwarz iteration k >= 1 in control-point space.
template <typename T>
void run_step(mfa_model* md) {
  mfa_handle* h = md->h;
  const LayoutDev& L = md->L;
  const int ns = md->nsub;
  T* S1 = (T*)md->S1;
  T* S2 = (T*)md->S2;
  auto opsk = [&](int kind) { return md->ops + (size_t)kind * ns; };
  std::swap(md->P, md->Pprev);  // Pprev <- P^{k-1}
  if constexpr (std::is_same<T, ff>::value) {
    if (md->dim == 3 && md->use_fused) {
      bool fused = false;
      TRACED(h, TR_SOLVE_U,
             fused = launch_schwarz3d_ff(L, md->offL, md->maxnL, md->maxnU, (const ff*)md->Pprev, (const ff*)md->BL,
                                         (ff*)md->X, h->stream));
      if (fused) {
        TRACED_N(h, TR_AVERAGE, 1,
                 launch_average_ff(L, md->offL, (const ff*)md->X, (ff*)md->P, (const ff*)md->Pprev, md->part,
                                   h->d_metrics, h->stream, md->update));
        return;
      }
    }
  }
  if (md->plain) {
    // the comparator form re-reads the data of every window each iteration
    if (md->q_src_dtype == MFA_F64)
      plain_project<T, double>(md, (const double*)md->q_src);
    else
      plain_project<T, float>(md, (const float*)md->q_src);
  }
  TRACED(h, TR_FRAME_GATHER, launch_frame_gather<T>(L, md->offS2, md->maxL, (const T*)md->Pprev, S2, h->stream));
  for (int a = 0; a < md->dim; ++a) {
    const T* in = (a % 2 == 0) ? S2 : S1;
    T* out = (a % 2 == 0) ? S1 : S2;
    if (md->plain) {
      for (int sd = 0; sd < ns; ++sd)
        TRACED(h, TR_BAND_APPLY,
               launch_band_apply<T>(L, a, opsk(OP_APPLY0 + a) + sd, 1, md->maxApply[a], in, out, h->stream));
    } else {
      TRACED(h, TR_BAND_APPLY,
             launch_band_apply<T>(L, a, opsk(OP_APPLY0 + a), ns, md->maxApply[a], in, out, h->stream));
    }
  }
  const T* Y = (md->dim % 2 == 1) ? S1 : S2;
  const long long* offY = (md->dim % 2 == 1) ? md->offS1 : md->offS2;
  TRACED(h, TR_RHS_FINALIZE,
         launch_rhs_finalize<T>(L, md->offL, offY, md->maxU, (const T*)md->BL, Y, (T*)md->X, h->stream));
  for (int a = 0; a < md->dim; ++a) {
    if (md->plain) {
      for (int sd = 0; sd < ns; ++sd)
        TRACED(h, TR_SOLVE_U,
               launch_band_solve<T>(L, a, true, opsk(OP_SOLVEU0 + a) + sd, 1, md->maxFibU[a], (T*)md->X, h->stream));
    } else {
      TRACED(h, TR_SOLVE_U,
             launch_band_solve<T>(L, a, true, opsk(OP_SOLVEU0 + a), ns, md->maxFibU[a], (T*)md->X, h->stream));
    }
  }
  cudaMemsetAsync(h->d_metrics, 0, 4 * sizeof(unsigned long long), h->stream);
  TRACED(h, TR_AVERAGE,
         launch_average<T>(L, md->offL, (const T*)md->X, (T*)md->P, (const T*)md->Pprev, h->d_metrics, h->stream,
                           md->update));
}

// Global grid decode; the last axis either writes `out` (type T) or is fused
// with the residual against q.
template <typename T, typename TQ, typename TOut>
int run_decode_grid(mfa_model* md, TOut* out, const TQ* q) {
  mfa_handle* h = md->h;
  const LayoutDev& L = md->L;
  const int ns = md->nsub;
  const int d = md->dim;
  // fused 3-D tiles: one kernel, residual partials per tile (FP32 data; FP64
  // data take the per-axis residual, which keeps them exact)
  if constexpr (std::is_same<T, ff>::value) {
    if (d == 3 && md->use_fused) {
      bool fused = false;
      if (q) {
        if constexpr (std::is_same<TQ, float>::value) {
          const long long tiles = decode3d_tiles(L);
          int rc = ensure_ws(h, (size_t)tiles * 4 * sizeof(double));
          if (rc != MFA_OK) return rc;
          double* part = (double*)h->ws;
          TRACED(h, TR_RESIDUAL,
                 fused = (launch_decode3d<ff, TQ, float, true>(L, (const ff*)md->P, q, nullptr, part, h->stream)));
          if (fused) {
            TRACED_N(h, TR_REDUCE, 2,
                     launch_reduce_partials(part, (int)tiles, h->d_result, h->stream, h->d_partials, kResidualBlocks));
            return MFA_OK;
          }
        }
      } else if constexpr (!std::is_same<TOut, ff>::value) {
        TRACED(h, TR_DECODE_OUT,
               fused = (launch_decode3d<ff, float, TOut, false>(L, (const ff*)md->P, (const float*)nullptr, out,
                                                                 nullptr, h->stream)));
        if (fused) return MFA_OK;
      }
    }
  }
  // scratch for intermediate stages
  long long sz[3] = {0, 0, 0};
  {
    long long cur[3] = {md->axh[0].n, md->axh[1].n, md->axh[2].n};
    for (int a = 0; a < d; ++a) {
      cur[a] = md->axh[a].M;
      sz[a] = cur[0] * cur[1] * cur[2];
    }
  }
  size_t need = 0;
  if (d >= 2) need += align256(sz[0] * sizeof(T));
  if (d >= 3) need += align256(sz[1] * sizeof(T));
  int rc = ensure_ws(h, std::max<size_t>(need, 256));
  if (rc != MFA_OK) return rc;
  T* bufA = (T*)h->ws;
  T* bufB = (T*)((char*)h->ws + align256(sz[0] * sizeof(T)));
  const T* in = (const T*)md->P;
  for (int a = 0; a < d; ++a) {
    const AxisOp* op = md->ops + (size_t)(OP_DEC0 + a) * ns;
    const bool last = a == d - 1;
    if (last) {
      if (q) {
        TRACED(h, TR_RESIDUAL,
               (launch_expand_residual<T, TQ>(L, a, op, sz[a], in, q, h->d_partials, kResidualBlocks, h->stream)));
        TRACED(h, TR_REDUCE, launch_reduce_partials(h->d_partials, kResidualBlocks, h->d_result, h->stream));
      } else {
        TRACED(h, TR_DECODE_OUT, (launch_expand<T, TOut>(L, a, op, 1, sz[a], in, out, h->stream)));
      }
    } else {
      T* o = (a == 0) ? bufA : bufB;
      TRACED(h, TR_DECODE_STAGE, (launch_expand<T, T>(L, a, op, 1, sz[a], in, o, h->stream)));
      in = o;
    }
  }
  return MFA_OK;
}

// One-sided derivatives of orders 0..R, with respect to the knot coordinate
// x = u * gspans, of the p+1 basis functions of axis `ax` nonzero next to the
// breakpoint xb (an integer knot position): on the span ending at xb (side 0,
// the left limit) or starting there (side 1, the right limit).  The degree is
// raised by the Cox-de Boor recurrence on the axis's own knot vector and the
// derivative orders come from
//   d/dx N_{m,q} = q/(t_{m+q}-t_m) N_{m,q-1} - q/(t_{m+q+1}-t_{m+1}) N_{m+1,q-1}
// (terms with a zero denominator dropped); with weights, the rational basis
// and its derivatives by the Leibniz rule.  out[r*(p+1) + c] is order r of
// control point first + c; returns first, or -1 if xb is not inside the axis.
int host_onesided_basis(const AxisHost& ax, int xb, int side, int R, double* out) {
  const int p = ax.p;
  const std::vector<int>& t = ax.knots;
  int i = -1;  // knot interval [t_i, t_{i+1}) with t_i < t_{i+1}
  for (int k = p; k + 1 < (int)t.size() - p; ++k) {
    if (t[k] >= t[k + 1]) continue;
    if ((side == 1 && t[k] == xb) || (side == 0 && t[k + 1] == xb)) {
      i = k;
      break;
    }
  }
  if (i < 0) return -1;
  const double x = xb;
  std::vector<double> D((size_t)(R + 1) * (p + 1), 0.0);
  for (int r = 0; r <= R; ++r) {
    double N[MFA_MAX_DEGREE + 1] = {0};
    if (r > p) continue;
    N[0] = 1.0;
    const int q0 = p - r;
    for (int q = 1; q <= p; ++q) {
      double nw[MFA_MAX_DEGREE + 1] = {0};
      for (int c = 0; c <= q; ++c) {
        const int m = i - q + c;  // function N_{m,q}; N_{m,q-1} = N[c-1], N_{m+1,q-1} = N[c]
        const double dl = t[m + q] - t[m], dr = t[m + q + 1] - t[m + 1];
        double v = 0.0;
        if (q <= q0) {
          if (c >= 1 && dl > 0) v += (x - t[m]) / dl * N[c - 1];
          if (c < q && dr > 0) v += (t[m + q + 1] - x) / dr * N[c];
        } else {
          if (c >= 1 && dl > 0) v += q / dl * N[c - 1];
          if (c < q && dr > 0) v -= q / dr * N[c];
        }
        nw[c] = v;
      }
      for (int c = 0; c <= q; ++c) N[c] = nw[c];
    }
    for (int c = 0; c <= p; ++c) D[(size_t)r * (p + 1) + c] = N[c];
  }
  const int first = i - p;
  if (!ax.wts.empty()) {
    std::vector<double> w(R + 1, 0.0);
    for (int r = 0; r <= R; ++r)
      for (int c = 0; c <= p; ++c) {
        D[(size_t)r * (p + 1) + c] *= ax.wts[first + c];
        w[r] += D[(size_t)r * (p + 1) + c];
      }
    for (int r = 0; r <= R; ++r) {
      double binom = 1.0;
      for (int j = 1; j <= r; ++j) {
        binom = binom * (r - j + 1) / j;
        for (int c = 0; c <= p; ++c) D[(size_t)r * (p + 1) + c] -= binom * w[j] * D[(size_t)(r - j) * (p + 1) + c];
      }
      for (int c = 0; c <= p; ++c) D[(size_t)r * (p + 1) + c] /= w[0];
    }
  }
  std::copy(D.begin(), D.end(), out);
  return first;
}

// Decoded error of the model's current P against device data qd: fills
// r = {sum E^2, max |E|, min Q, max Q}; synchronous.
int model_residual(mfa_model* md, const void* qd, int q_dtype, double r[4]) {
  mfa_handle* h = md->h;
  int rc;
  if (md->prec == MFA_PREC_FP64)
    rc = q_dtype == MFA_F64 ? run_decode_grid<double, double, double>(md, nullptr, (const double*)qd)
                            : run_decode_grid<double, float, double>(md, nullptr, (const float*)qd);
  else
    rc = q_dtype == MFA_F64 ? run_decode_grid<ff, double, ff>(md, nullptr, (const double*)qd)
                            : run_decode_grid<ff, float, ff>(md, nullptr, (const float*)qd);
  if (rc != MFA_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(h->h_pinned, h->d_result, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  std::memcpy(r, h->h_pinned, 4 * sizeof(double));
  return MFA_OK;
}

int read_status(mfa_handle* h) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(h->h_pinned, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  std::memcpy(&st, h->h_pinned, sizeof(int));
  if (st != 0) cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* mfa_status_string(int s) {
  switch (s) {
    case MFA_OK: return "ok";
    case MFA_NOT_CONVERGED: return "not converged (max_iters reached)";
    case MFA_ERR_ARG: return "invalid argument";
    case MFA_ERR_LAYOUT: return "invalid layout";
    case MFA_ERR_OOM: return "device out of memory";
    case MFA_ERR_CUDA: return "CUDA error";
    case MFA_ERR_NOT_SPD: return "local normal matrix not positive definite";
    case MFA_ERR_DIVERGED: return "Schwarz iteration diverged";
    case MFA_ERR_NONFINITE: return "non-finite input data";
    case MFA_ERR_UNSUPPORTED: return "unsupported request";
    case MFA_ERR_TIMEOUT: return "device wait on an asynchronous copy timed out";
    case MFA_ERR_IO: return "file could not be read or written, or is not a saved model";
    default: return "unknown status";
  }
}

int mfa_axis_layout(int64_t npts, int32_t nspans, int32_t degree, int32_t nsub, const int32_t* core_spans,
                    int32_t overlap, int32_t knots, int32_t* out, int32_t cap, int32_t* owner) {
  if (!out || npts < 1 || degree < 1 || degree > MFA_MAX_DEGREE || nsub < 1 || cap < nsub) return MFA_ERR_ARG;
  AxisHost ax;
  const int rc = build_axis(ax, npts, nspans, degree, nsub, core_spans, overlap, knots);
  if (rc != MFA_OK) return rc;
  for (int s = 0; s < nsub; ++s) {
    const AxisSub& sb = ax.subs[s];
    int32_t* o = out + 10 * (size_t)s;
    o[8] = sb.oU;
    o[9] = sb.nU;
    o[0] = sb.a;
    o[1] = sb.b;
    o[2] = sb.w0;
    o[3] = sb.w1;
    o[4] = sb.k0;
    o[5] = sb.k0 + sb.m - 1;
    o[6] = sb.l0;
    o[7] = sb.nL;
  }
  if (owner)
    for (int g = 0; g < ax.n; ++g) owner[g] = ax.own_first[g] + ax.own_pick[g];
  return MFA_OK;
}

int mfa_create(int device, void* cuda_stream, mfa_handle** out) {
  if (!out) return MFA_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MFA_ERR_ARG;
  }
  DeviceGuard g(device);
  mfa_handle* h = new (std::nothrow) mfa_handle();
  if (!h) return MFA_ERR_OOM;
  h->device = device;
  h->stream = (cudaStream_t)cuda_stream;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaError_t e = cudaMemPoolCreate(&h->pool, &props);
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_metrics, 256);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_partials, 4 * sizeof(double) * kResidualBlocks);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_result, 256);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_pinned, 256);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->stage32_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->rb_done, cudaEventDisableTiming);
  for (int i = 0; i <= kSlabs && e == cudaSuccess; ++i) {
    cudaEvent_t ev = nullptr;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) h->slab_ev.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, 256, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mfa_destroy(h);
    return cuda_status(e);
  }
  *out = h;
  return MFA_OK;
}

int mfa_destroy(mfa_handle* h) {
  if (!h) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  if (h->ws) cudaFreeAsync(h->ws, h->stream);
  if (h->rb) cudaFreeAsync(h->rb, h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->pool) cudaMemPoolDestroy(h->pool);
  cudaFree(h->d_status);
  cudaFree(h->d_metrics);
  cudaFree(h->d_partials);
  cudaFree(h->d_result);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  if (h->stage_done) cudaEventDestroy(h->stage_done);
  if (h->h_stage32) cudaFreeHost(h->h_stage32);
  if (h->stage32_done) cudaEventDestroy(h->stage32_done);
  for (cudaEvent_t ev : h->slab_ev) cudaEventDestroy(ev);
  if (h->rb_ready) cudaEventDestroy(h->rb_ready);
  if (h->rb_done) cudaEventDestroy(h->rb_done);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->plan && h->plan_free) h->plan_free(h->plan);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  delete h;
  return MFA_OK;
}

namespace {
// Offsets of a model's device tables (one arena: the host-filled tables
// first, then those the setup kernels compute) and buffers (one pool block).
struct TablePlan {
  size_t o_w[3];
  size_t o_span[3], o_vd[3], o_vf[3], o_vff[3], o_ss[3], o_subs[3], o_of[3], o_oc[3], o_AL[3], o_fLd[3], o_fLf[3],
      o_fLff[3], o_fUd[3], o_fUf[3], o_fUff[3], o_ot[3], o_nlt[3], o_pk[3], o_one[3];
  size_t o_offL = 0, o_offS1 = 0, o_offS2 = 0, o_ops = 0, o_rows = 0, o_xs = 0;
  int n_full_rows = 0, n_part_rows = 0, n_xs = 0;
  size_t host_bytes = 0, tables_bytes = 0;
  size_t o_BL = 0, o_X = 0, o_P = 0, o_Pp = 0, o_S1 = 0, o_S2 = 0, o_part = 0, o_stage = 0, big_bytes = 0;
  size_t o_zpart = 0, o_zctr = 0, o_units = 0;
};

// Host products of one layout, kept per handle for the most recent layout of
// a single model: the host axes and operand tables (a model copy without
// device memory) and the table plan, whose image stays in h->h_stage while
// h->plan_valid.  A model of the same layout then skips the host build; every
// kernel (setup included) still runs.
struct PlanCache {
  mfa_layout lay{};
  std::vector<int32_t> cores[3];
  std::vector<double> wts[3];
  bool plain = false;
  size_t stage_bytes = 0;
  mfa_model* proto = nullptr;
  TablePlan tp;
};

bool plan_matches(const PlanCache& pc, const mfa_layout* lay, bool plain, size_t stage_bytes) {
  if (pc.plain != plain || pc.stage_bytes != stage_bytes) return false;
  const mfa_layout& k = pc.lay;
  if (k.dim != lay->dim || k.degree != lay->degree || k.precision != lay->precision || k.knots != lay->knots)
    return false;
  for (int a = 0; a < lay->dim && a < 3; ++a) {
    if (k.npts[a] != lay->npts[a] || k.nspans[a] != lay->nspans[a] || k.nsub[a] != lay->nsub[a] ||
        k.overlap[a] != lay->overlap[a] || k.lo[a] != lay->lo[a] || k.hi[a] != lay->hi[a])
      return false;
    if ((lay->core_spans[a] == nullptr) != pc.cores[a].empty()) return false;
    if (lay->core_spans[a] &&
        std::memcmp(lay->core_spans[a], pc.cores[a].data(), sizeof(int32_t) * pc.cores[a].size()) != 0)
      return false;
    if ((lay->weights[a] == nullptr) != pc.wts[a].empty()) return false;
    if (lay->weights[a] && std::memcmp(lay->weights[a], pc.wts[a].data(), sizeof(double) * pc.wts[a].size()) != 0)
      return false;
  }
  return true;
}

// Allocate the model's tables and buffers, upload the host-filled tables from
// the handle's pinned image (h->h_stage, host_bytes long), fill the device
// layout and run the setup kernels (basis, Gram bands, Cholesky factors).
int bind_model(mfa_handle* h, mfa_model* md, const TablePlan& tp) {
  int rc = pool_alloc(h, &md->arena, tp.tables_bytes);
  if (rc == MFA_OK) rc = pool_alloc(h, &md->big, tp.big_bytes);
  if (rc != MFA_OK) {
    pool_free(h, md->arena);
    pool_free(h, md->big);
    md->arena = md->big = nullptr;
    return rc;
  }
  // pinned source: the copy runs ahead of the setup kernels on the stream
  cudaError_t e = cudaMemcpyAsync(md->arena, h->h_stage, tp.host_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->stage_done, h->stream);
  LayoutDev& L = md->L;
  L.dim = md->dim;
  L.nsub = md->nsub;
  for (int a = 0; a < 3; ++a) {
    const AxisHost& ax = md->axh[a];
    L.S[a] = ax.S;
    L.ncp[a] = ax.n;
    L.M[a] = ax.M;
    AxisDev& d = L.ax[a];
    d.M = ax.M;
    d.nspans = ax.nspans;
    d.p = ax.p;
    d.n = ax.n;
    d.S = ax.S;
    d.pieces = ax.pieces;
    d.kmode = ax.kmode;
    d.gspans = ax.gspans;
    d.wts = ax.wts.empty() ? nullptr : at_off<double>(md->arena, tp.o_w[a]);
    d.span = at_off<int>(md->arena, tp.o_span[a]);
    d.vals_d = at_off<double>(md->arena, tp.o_vd[a]);
    d.vals_f = at_off<float>(md->arena, tp.o_vf[a]);
    d.vals_ff = at_off<ff>(md->arena, tp.o_vff[a]);
    d.span_start = at_off<int>(md->arena, tp.o_ss[a]);
    d.subs = at_off<AxisSub>(md->arena, tp.o_subs[a]);
    d.own_first = at_off<int>(md->arena, tp.o_of[a]);
    d.own_count = at_off<int>(md->arena, tp.o_oc[a]);
    d.own_tab = at_off<int4>(md->arena, tp.o_ot[a]);
    d.nL_tab = at_off<int>(md->arena, tp.o_nlt[a]);
    d.own_pick = at_off<int>(md->arena, tp.o_pk[a]);
    d.one_rng = at_off<int2>(md->arena, tp.o_one[a]);
    d.AL = at_off<double>(md->arena, tp.o_AL[a]);
    d.facL_d = at_off<double>(md->arena, tp.o_fLd[a]);
    d.facL_f = at_off<float>(md->arena, tp.o_fLf[a]);
    d.facL_ff = at_off<ff>(md->arena, tp.o_fLff[a]);
    d.facU_d = at_off<double>(md->arena, tp.o_fUd[a]);
    d.facU_f = at_off<float>(md->arena, tp.o_fUf[a]);
    d.facU_ff = at_off<ff>(md->arena, tp.o_fUff[a]);
  }
  L.shared_rows = at_off<int>(md->arena, tp.o_rows);
  L.n_full_rows = tp.n_full_rows;
  L.n_part_rows = tp.n_part_rows;
  L.shared_x = at_off<int>(md->arena, tp.o_xs);
  L.n_shared_x = tp.n_xs;
  md->offL = at_off<long long>(md->arena, tp.o_offL);
  md->offS1 = at_off<long long>(md->arena, tp.o_offS1);
  md->offS2 = at_off<long long>(md->arena, tp.o_offS2);
  md->ops = at_off<AxisOp>(md->arena, tp.o_ops);
  md->BL = at_off<char>(md->big, tp.o_BL);
  md->X = at_off<char>(md->big, tp.o_X);
  md->P = at_off<char>(md->big, tp.o_P);
  md->Pprev = at_off<char>(md->big, tp.o_Pp);
  md->S1 = at_off<char>(md->big, tp.o_S1);
  md->S2 = at_off<char>(md->big, tp.o_S2);
  md->part = at_off<float>(md->big, tp.o_part);
  md->zpart = md->zsplit > 1 ? at_off<ff>(md->big, tp.o_zpart) : nullptr;
  md->units = md->zsplit > 1 ? at_off<int2>(md->arena, tp.o_units) : nullptr;
  md->zctr = md->zsplit > 1 ? at_off<unsigned>(md->big, tp.o_zctr) : nullptr;
  // setup kernels: basis tables, Gram bands, Cholesky factors (FP64), all axes per launch
  {
    int maxnL = 1;
    for (int a = 0; a < 3; ++a) maxnL = std::max(maxnL, md->maxnL[a]);
    TRACED_N(h, TR_SETUP, 2, launch_setup_all(L.ax, 3, maxnL, h->d_status, h->stream));
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    pool_free(h, md->arena);
    pool_free(h, md->big);
    md->arena = md->big = nullptr;
    return cuda_status(e);
  }
  return MFA_OK;
}

// Upload the layout tables of a model whose host axes (md->axh) and operand
// tables are built, allocate its buffers (plus `stage_bytes` for staged host
// data, offset returned in *o_stage), fill the device layout and run the
// setup kernels.  The table image is built in the handle's pinned staging
// buffer; the plan is returned in *keep when given.
int materialize_model(mfa_handle* h, mfa_model* md, const std::vector<AxisOp>& ops,
                      const std::vector<long long>& offL, const std::vector<long long>& offS1,
                      const std::vector<long long>& offS2, size_t stage_bytes, size_t* o_stage,
                      TablePlan* keep = nullptr) {
  const int ns = md->nsub;
  TablePlan tp;
  Arena ar;
  // fused projection: four units per window along z (whole batches of
  // planes) when every unit keeps more than p+1 knot spans, so that a
  // z-control point takes planes of two units at most; partial sums of the
  // shared z-control points (p+1 per side of a cut)
  md->zsplit = 1;
  if (!md->batch && md->dim == 3 && md->prec == MFA_PREC_MIXED && md->use_fused) {
    const AxisHost& az = md->axh[2];
    constexpr int kUnits = 4;
    const int zb = proj3d_planes_per_batch(md->degree, md->maxm[0], md->maxm[1], md->maxm[2], md->maxnL[0],
                                           md->maxnL[1]);
    bool ok = true;
    for (const AxisSub& sb : az.subs)
      ok = ok && proj3d_split_ok(az.p, zb, kUnits, az.M, az.nspans, sb.k0, sb.m);
    if (ok) md->zsplit = kUnits;
  }
  // the projection units ordered by the slab of host data their last plane
  // lies in (slab t: planes [t sp, (t+1) sp) of the grid), so that the units
  // of slab t can run as soon as slabs 0..t have landed
  std::vector<int2> units;
  md->slab_units.assign(kSlabs + 1, 0);
  md->slab_planes = 0;
  if (md->zsplit > 1) {
    const AxisHost& az = md->axh[2];
    const int zb = proj3d_planes_per_batch(md->degree, md->maxm[0], md->maxm[1], md->maxm[2], md->maxnL[0],
                                           md->maxnL[1]);
    const long long sp = (az.M + kSlabs - 1) / kSlabs;
    md->slab_planes = sp;
    std::vector<std::vector<int2>> by_slab(kSlabs);
    for (int sd = 0; sd < ns; ++sd) {
      const AxisSub& sb = az.subs[sd / (md->axh[0].S * md->axh[1].S)];
      for (int k = 0; k < md->zsplit; ++k) {
        const long long end = sb.k0 + proj3d_unit_start(sb.m, zb, md->zsplit, k + 1);  // one past the last plane
        const int t = (int)std::min<long long>(kSlabs - 1, std::max<long long>(0, (end + sp - 1) / sp - 1));
        by_slab[t].push_back(int2{sd, k});
      }
    }
    for (int t = 0; t < kSlabs; ++t) {
      units.insert(units.end(), by_slab[t].begin(), by_slab[t].end());
      md->slab_units[t + 1] = (int)units.size();
    }
  }
  // tables filled on the host come first (one upload), then the ones the
  // setup kernels compute
  for (int a = 0; a < 3; ++a) {
    const AxisHost& ax = md->axh[a];
    tp.o_ss[a] = ar.take<int>(ax.nspans + 1);
    tp.o_subs[a] = ar.take<AxisSub>(ax.S);
    tp.o_of[a] = ar.take<int>(ax.n);
    tp.o_oc[a] = ar.take<int>(ax.n);
    tp.o_ot[a] = ar.take<int4>(ax.n);
    tp.o_nlt[a] = ar.take<int>(ax.S);
    tp.o_pk[a] = ar.take<int>(ax.n);
    tp.o_one[a] = ar.take<int2>(ax.S);
    tp.o_w[a] = ar.take<double>(ax.wts.size());
  }
  tp.o_offL = ar.take<long long>(ns);
  tp.o_offS1 = ar.take<long long>(ns);
  tp.o_offS2 = ar.take<long long>(ns);
  tp.o_ops = ar.take<AxisOp>(ops.size());
  // rows of control points with two owners on some axis (float-float update):
  // rows with two owners along y or z first, then the rest with the x
  // positions that have two owners
  std::vector<int> rows_full, rows_part, xs;
  if (!md->batch) {  // axes beyond the dimension have one control point with one owner
    const AxisHost &a0 = md->axh[0], &a1 = md->axh[1], &a2 = md->axh[2];
    for (int g0 = 0; g0 < a0.n; ++g0)
      if (a0.own_count[g0] == 2) xs.push_back(g0);
    for (int g2 = 0; g2 < a2.n; ++g2)
      for (int g1 = 0; g1 < a1.n; ++g1) {
        const int r = g1 + a1.n * g2;
        if (a1.own_count[g1] == 2 || a2.own_count[g2] == 2)
          rows_full.push_back(r);
        else if (!xs.empty())
          rows_part.push_back(r);
      }
  }
  tp.o_units = ar.take<int2>(units.size());
  tp.o_rows = ar.take<int>(rows_full.size() + rows_part.size());
  tp.o_xs = ar.take<int>(xs.size());
  tp.n_full_rows = (int)rows_full.size();
  tp.n_part_rows = (int)rows_part.size();
  tp.n_xs = (int)xs.size();
  tp.host_bytes = ar.used;
  for (int a = 0; a < 3; ++a) {
    const AxisHost& ax = md->axh[a];
    const int w = ax.p + 1;
    tp.o_span[a] = ar.take<int>(ax.M);
    tp.o_vd[a] = ar.take<double>((size_t)ax.M * w);
    tp.o_vf[a] = ar.take<float>((size_t)ax.M * w);
    tp.o_vff[a] = ar.take<ff>((size_t)ax.M * w);
    tp.o_AL[a] = ar.take<double>((size_t)ax.bandL_rows * w);
    tp.o_fLd[a] = ar.take<double>((size_t)ax.bandL_rows * w);
    tp.o_fLf[a] = ar.take<float>((size_t)ax.bandL_rows * w);
    tp.o_fLff[a] = ar.take<ff>((size_t)ax.bandL_rows * w);
    tp.o_fUd[a] = ar.take<double>((size_t)ax.bandU_rows * w);
    tp.o_fUf[a] = ar.take<float>((size_t)ax.bandU_rows * w);
    tp.o_fUff[a] = ar.take<ff>((size_t)ax.bandU_rows * w);
  }
  tp.tables_bytes = ar.used;
  // big buffers
  const size_t es = elem_size(md->prec);
  Arena bg;
  // a batch group writes B_L and X into the batch's buffers and has no global P
  const long long own_sizeL = md->batch ? 0 : md->sizeL;
  tp.o_BL = bg.take<char>(own_sizeL * es);
  tp.o_X = bg.take<char>(own_sizeL * es);
  const long long ncp = md->batch ? 0 : (long long)md->axh[0].n * md->axh[1].n * md->axh[2].n;
  tp.o_P = bg.take<char>(ncp * es);
  tp.o_Pp = bg.take<char>(ncp * es);
  tp.o_S1 = bg.take<char>(md->sizeS1 * es);
  tp.o_S2 = bg.take<char>(md->sizeS2 * es);
  // update partials (3 floats per block of the float-float update), its row
  // counter and its finished-block counter
  tp.o_part = bg.take<float>(3 * (size_t)(ns + kAvgListBlocks) + 2);
  if (md->zsplit > 1) {
    tp.o_zpart =
        bg.take<ff>((size_t)ns * (md->zsplit - 1) * 2 * (md->degree + 1) * md->maxnL[0] * md->maxnL[1]);
    tp.o_zctr = bg.take<unsigned>(ns);
  }
  // host data staging: the data are copied into the pool before use
  tp.o_stage = stage_bytes ? bg.take<char>(stage_bytes) : 0;
  tp.big_bytes = bg.used;
  // host image of the uploaded tables, built in the handle's pinned staging
  // buffer once its previous upload has been read (alignment gaps are never
  // read, so the image is not cleared); it no longer holds a cached plan
  h->plan_valid = false;
  cudaEventSynchronize(h->stage_done);
  if (h->h_stage_cap < tp.host_bytes) {
    if (h->h_stage) cudaFreeHost(h->h_stage);
    h->h_stage = nullptr;
    h->h_stage_cap = 0;
    if (cudaMallocHost(&h->h_stage, tp.host_bytes) != cudaSuccess) {
      cudaGetLastError();
      h->h_stage = nullptr;
      return MFA_ERR_OOM;
    }
    h->h_stage_cap = tp.host_bytes;
  }
  char* img = h->h_stage;
  for (int a = 0; a < 3; ++a) {
    const AxisHost& ax = md->axh[a];
    std::memcpy(img + tp.o_ss[a], ax.span_start.data(), sizeof(int) * ax.span_start.size());
    std::memcpy(img + tp.o_subs[a], ax.subs.data(), sizeof(AxisSub) * ax.subs.size());
    std::memcpy(img + tp.o_of[a], ax.own_first.data(), sizeof(int) * ax.n);
    std::memcpy(img + tp.o_oc[a], ax.own_count.data(), sizeof(int) * ax.n);
    std::memcpy(img + tp.o_ot[a], ax.own_tab.data(), sizeof(int4) * ax.n);
    std::memcpy(img + tp.o_nlt[a], ax.nL_tab.data(), sizeof(int) * ax.S);
    std::memcpy(img + tp.o_pk[a], ax.own_pick.data(), sizeof(int) * ax.n);
    std::memcpy(img + tp.o_one[a], ax.one_rng.data(), sizeof(int2) * ax.S);
    std::memcpy(img + tp.o_w[a], ax.wts.data(), sizeof(double) * ax.wts.size());
  }
  std::memcpy(img + tp.o_rows, rows_full.data(), sizeof(int) * rows_full.size());
  std::memcpy(img + tp.o_rows + sizeof(int) * rows_full.size(), rows_part.data(), sizeof(int) * rows_part.size());
  std::memcpy(img + tp.o_xs, xs.data(), sizeof(int) * xs.size());
  std::memcpy(img + tp.o_units, units.data(), sizeof(int2) * units.size());
  std::memcpy(img + tp.o_offL, offL.data(), sizeof(long long) * ns);
  std::memcpy(img + tp.o_offS1, offS1.data(), sizeof(long long) * ns);
  std::memcpy(img + tp.o_offS2, offS2.data(), sizeof(long long) * ns);
  std::memcpy(img + tp.o_ops, ops.data(), sizeof(AxisOp) * ops.size());
  *o_stage = tp.o_stage;
  if (keep) *keep = tp;
  return bind_model(h, md, tp);
}
}  // namespace

namespace {
int encode_impl(mfa_handle* h, const mfa_layout* lay, const void* q, int q_dtype, int q_on_device, bool plain,
                mfa_model** out);
}

int mfa_encode(mfa_handle* h, const mfa_layout* lay, const void* q, int q_dtype, int q_on_device, mfa_model** out) {
  return encode_impl(h, lay, q, q_dtype, q_on_device, false, out);
}

int mfa_encode_plain(mfa_handle* h, const mfa_layout* lay, const void* q, int q_dtype, int q_on_device,
                     int32_t max_iters, double tol_dP, mfa_report* rep, mfa_model** out) {
  if (!h || !lay || !out || max_iters < 0) return MFA_ERR_ARG;
  if (lay->precision != MFA_PREC_FP64) return MFA_ERR_ARG;
  int rc = encode_impl(h, lay, q, q_dtype, q_on_device, true, out);
  if (rc != MFA_OK) return rc;
  rc = mfa_schwarz_iterate(h, *out, max_iters, tol_dP, 0.0, rep);
  if (rc < 0) {
    mfa_free(*out);
    *out = nullptr;
  }
  return rc;
}

namespace {
// A model for a layout: host layout, operand tables, device tables, buffers
// (plus stage_bytes for staged host data, offset in *o_stage) and the setup
// kernels (basis, Gram bands, Cholesky factors).  No data are read.
int create_model(mfa_handle* h, const mfa_layout* lay, bool plain, size_t stage_bytes, mfa_model** out,
                 size_t* o_stage) {
  *out = nullptr;
  if (lay->dim < 1 || lay->dim > MFA_MAX_DIM) return MFA_ERR_ARG;
  if (lay->degree < 1 || lay->degree > MFA_MAX_DEGREE) return MFA_ERR_ARG;
  if (lay->precision != MFA_PREC_FP64 && lay->precision != MFA_PREC_MIXED) return MFA_ERR_ARG;
  if (lay->knots != MFA_KNOTS_FLOATING && lay->knots != MFA_KNOTS_CLAMPED) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  if (h->plan_valid && h->plan && h->plan->proto && plan_matches(*h->plan, lay, plain, stage_bytes)) {
    mfa_model* md = new (std::nothrow) mfa_model(*h->plan->proto);
    if (!md) return MFA_ERR_OOM;
    const int rc = bind_model(h, md, h->plan->tp);
    if (rc != MFA_OK) {
      delete md;
      return rc;
    }
    *o_stage = h->plan->tp.o_stage;
    *out = md;
    return MFA_OK;
  }
  mfa_model* md = new (std::nothrow) mfa_model();
  if (!md) return MFA_ERR_OOM;
  md->h = h;
  md->plain = plain;
  if (plain) md->use_fused = false;
  md->prec = lay->precision;
  md->dim = lay->dim;
  md->degree = lay->degree;
  long long npts_total = 1;
  for (int a = 0; a < 3; ++a) {
    int rc;
    if (a < lay->dim) {
      if (lay->npts[a] < 1) {
        delete md;
        return MFA_ERR_ARG;
      }
      rc = build_axis(md->axh[a], lay->npts[a], lay->nspans[a], lay->degree, lay->nsub[a], lay->core_spans[a],
                      lay->overlap[a], lay->knots);
      if (rc == MFA_OK && lay->weights[a]) {
        // separable NURBS weights (Sec. 2.1, Eq. nurbs-basis): positive and finite
        AxisHost& ax = md->axh[a];
        ax.wts.assign(lay->weights[a], lay->weights[a] + ax.n);
        for (double w : ax.wts)
          if (!(w > 0.0) || !std::isfinite(w)) rc = MFA_ERR_ARG;
      }
      md->lo[a] = lay->lo[a];
      md->hi[a] = lay->hi[a];
      md->overlap[a] = lay->overlap[a];
      npts_total *= lay->npts[a];
    } else {
      rc = build_axis(md->axh[a], 1, 1, 0, 1, nullptr, 0);
    }
    if (rc != MFA_OK) {
      delete md;
      return rc;
    }
  }
  if (npts_total > (1LL << 40)) {
    delete md;
    return MFA_ERR_ARG;
  }
  md->nsub = md->axh[0].S * md->axh[1].S * md->axh[2].S;
  md->knots = lay->knots;
  for (int a = 0; a < 3; ++a)
    if (md->axh[a].kmode != KMODE_FLOATING) md->use_fused = false;  // the fused kernels take uniform spans
  {
    // the fused projection's stage-1 output of control point c (floats
    // 4(c/2) + c%2 and 4(c/2) + c%2 + 2 of the staged row) is written while
    // the 16-byte chunk holding the first point of span c+1 is in registers;
    // it must not reach past that chunk; and consecutive points advance at
    // most one span (stage 1 emits at most one control point per point)
    const AxisHost& ax = md->axh[0];
    for (const AxisSub& sb : ax.subs) {
      long long prev = -1;
      for (int k = 0; k < sb.m && md->x_inplace_ok; ++k) {
        const long long gk = sb.k0 + k;
        long long sk = ax.M == 1 ? 0 : (gk * ax.nspans) / (ax.M - 1);
        if (sk > ax.nspans - 1) sk = ax.nspans - 1;
        const long long cmax = sk - sb.l0 - 1;  // highest CP emitted before reading point k
        if (cmax >= 0 && stage1_reach(cmax) > 4 * (k / 4) + 3) md->x_inplace_ok = false;
        if (k > 0 && sk - prev > 1) md->x_inplace_ok = false;
        prev = sk;
      }
    }
  }
  std::vector<AxisOp> ops;
  std::vector<long long> offL, offS1, offS2;
  build_ops(md, ops, offL, offS1, offS2);
  TablePlan tp;
  int rc = materialize_model(h, md, ops, offL, offS1, offS2, stage_bytes, o_stage, &tp);
  if (rc != MFA_OK) {
    delete md;
    return rc;
  }
  // keep this layout's host products (no device memory) for its next model
  if (!h->plan) {
    h->plan = new (std::nothrow) PlanCache();
    h->plan_free = [](PlanCache* pc) {
      delete pc->proto;
      delete pc;
    };
  }
  if (h->plan) {
    PlanCache& pc = *h->plan;
    delete pc.proto;
    pc.proto = new (std::nothrow) mfa_model(*md);
    if (pc.proto) {
      pc.proto->arena = pc.proto->big = nullptr;
      pc.lay = *lay;
      for (int a = 0; a < 3; ++a) {
        pc.cores[a].clear();
        if (a < lay->dim && lay->core_spans[a]) pc.cores[a].assign(lay->core_spans[a], lay->core_spans[a] + lay->nsub[a]);
        pc.lay.core_spans[a] = nullptr;
        pc.wts[a] = a < lay->dim ? md->axh[a].wts : std::vector<double>();
        pc.lay.weights[a] = nullptr;
      }
      pc.plain = plain;
      pc.stage_bytes = stage_bytes;
      pc.tp = tp;
      h->plan_valid = true;
    }
  }
  *out = md;
  return MFA_OK;
}

int encode_impl(mfa_handle* h, const mfa_layout* lay, const void* q, int q_dtype, int q_on_device, bool plain,
                mfa_model** out) {
  if (!h || !lay || !q || !out) return MFA_ERR_ARG;
  *out = nullptr;
  if (q_dtype != MFA_F32 && q_dtype != MFA_F64) return MFA_ERR_ARG;
  long long npts_total = 1;
  for (int a = 0; a < lay->dim && a < 3; ++a) npts_total *= std::max<long long>(lay->npts[a], 1);
  const size_t qbytes = (size_t)npts_total * (q_dtype == MFA_F64 ? 8 : 4);
  size_t o_Q = 0;
  mfa_model* md = nullptr;
  int rc = create_model(h, lay, plain, q_on_device ? 0 : qbytes, &md, &o_Q);
  if (rc != MFA_OK) return rc;
  DeviceGuard g(h->device);
  cudaError_t e = cudaSuccess;
  const void* qd = q;
  StagedCopy sc{};
  bool staged = false;
  if (!q_on_device) {
    void* qbuf = at_off<char>(md->big, o_Q);
    if (md->units && (int)h->slab_ev.size() > kSlabs) {
      // fused 3-D projection: the data cross in z-slabs on the copy stream
      // (once the staging buffer's allocation is ordered before them) and
      // the projection units of each slab start as it lands
      e = cudaEventRecord(h->slab_ev[kSlabs], h->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->slab_ev[kSlabs], 0);
      sc = StagedCopy{q, qbuf, (size_t)lay->npts[0] * lay->npts[1] * (q_dtype == MFA_F64 ? 8 : 4), lay->npts[2]};
      staged = true;
    } else {
      // host data: copy and wait, so the caller may reuse its buffer on return
      if (e == cudaSuccess) e = cudaMemcpyAsync(qbuf, q, qbytes, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    qd = qbuf;
    md->q_staged = qbuf;
    md->q_staged_dtype = q_dtype;
  }
  md->q_src = qd;
  md->q_src_dtype = q_dtype;
  const StagedCopy* scp = staged ? &sc : nullptr;
  if (md->prec == MFA_PREC_FP64) {
    if (q_dtype == MFA_F64)
      run_encode<double, double>(md, (const double*)qd, scp);
    else
      run_encode<double, float>(md, (const float*)qd, scp);
  } else {
    if (q_dtype == MFA_F64)
      run_encode<ff, double>(md, (const double*)qd, scp);
    else
      run_encode<ff, float>(md, (const float*)qd, scp);
  }
  // the copies of the host data have finished when this returns, so the
  // caller may reuse its buffer (the fit itself goes on on the stream); on
  // an error too, before the staging buffer is released
  if (staged) {
    const cudaError_t ec = cudaStreamSynchronize(h->copy_stream);
    if (e == cudaSuccess) e = ec;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    pool_free(h, md->arena);
    pool_free(h, md->big);
    delete md;
    return cuda_status(e);
  }
  md->iters = 0;
  md->has_state = true;
  h->live_models++;
  *out = md;
  return MFA_OK;
}
}  // namespace

int mfa_set_update_rule(mfa_handle* h, mfa_model* md, int rule) {
  if (!h || !md || md->h != h || md->batch) return MFA_ERR_ARG;
  if (rule != MFA_UPDATE_AVERAGE && rule != MFA_UPDATE_OWNER) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  md->update = rule == MFA_UPDATE_OWNER ? UPDATE_OWNER : UPDATE_AVERAGE;
  // redo the current update from the copies the model holds
  cudaMemsetAsync(h->d_metrics, 0, 4 * sizeof(unsigned long long), h->stream);
  if (md->prec == MFA_PREC_FP64)
    TRACED(h, TR_AVERAGE, launch_average<double>(md->L, md->offL, (const double*)md->X, (double*)md->P, nullptr,
                                                 h->d_metrics, h->stream, md->update));
  else if (md->use_fused)
    TRACED_N(h, TR_AVERAGE, 1, launch_average_ff(md->L, md->offL, (const ff*)md->X, (ff*)md->P, nullptr, md->part,
                                                 h->d_metrics, h->stream, md->update));
  else
    TRACED(h, TR_AVERAGE, launch_average<ff>(md->L, md->offL, (const ff*)md->X, (ff*)md->P, nullptr, h->d_metrics,
                                             h->stream, md->update));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int mfa_schwarz_iterate(mfa_handle* h, mfa_model* md, int32_t max_iters, double tol_dP, double tol_rms_stall,
                        mfa_report* rep) {
  if (!h || !md || md->h != h || max_iters < 0 || (!md->has_state && max_iters > 0)) return MFA_ERR_ARG;
  if (!(tol_rms_stall == tol_rms_stall) || !(tol_dP == tol_dP)) return MFA_ERR_ARG;
  const bool stall = tol_rms_stall > 0 && max_iters > 0;
  if (stall && (!md->q_src || md->batch)) return MFA_ERR_ARG;  // the stall test decodes against the encoded data
  DeviceGuard g(h->device);
  // encode-time device errors surface here, or with the first iteration's
  // metrics (one read-back per iteration carries both)
  int status = 0;
  if (max_iters == 0 || stall) {
    status = read_status(h);
    if (status < 0) return status;
  }
  const long long npts = (long long)md->axh[0].M * md->axh[1].M * md->axh[2].M;
  double res[4] = {0, 0, 0, 0};
  double rms_prev = 0.0;
  if (stall) {
    // RMS of the current iterate (P^0 right after the encode)
    const int rr = model_residual(md, md->q_src, md->q_src_dtype, res);
    if (rr != MFA_OK) return rr;
    rms_prev = std::sqrt(res[0] / (double)npts);
  }
  int rc = MFA_NOT_CONVERGED;
  for (int it = 0; it < max_iters; ++it) {
    if (md->prec == MFA_PREC_FP64)
      run_step<double>(md);
    else
      run_step<ff>(md);
    // the metrics and the status word in one read-back
    cudaError_t e = cudaMemcpyAsync(h->h_pinned, h->d_metrics, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->h_pinned + 4, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned long long bits[3];
    std::memcpy(bits, h->h_pinned, sizeof(bits));
    double v[3];
    std::memcpy(v, bits, sizeof(v));
    int st = 0;
    std::memcpy(&st, h->h_pinned + 4, sizeof(int));
    if (st != 0) {
      cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream);
      if (st < 0) {
        status = st;
        rc = st;
        break;
      }
    }
    const double dP = v[1] > 0 ? v[0] / v[1] : 0.0;
    md->iters++;
    if (md->iters > 1 && dP > md->last_dP && dP > 0)
      md->grow_streak++;
    else
      md->grow_streak = 0;
    md->last_dP = dP;
    md->last_jump = v[2];
    md->last_rms = -1.0;
    if (!std::isfinite(dP) || md->grow_streak >= 8) {
      rc = MFA_ERR_DIVERGED;
      break;
    }
    if (tol_dP > 0 && dP <= tol_dP) {
      rc = MFA_OK;
      break;
    }
    if (stall) {
      // decoded-residual stall: |RMS_k - RMS_{k-1}| <= tol * RMS_k
      const int rr = model_residual(md, md->q_src, md->q_src_dtype, res);
      if (rr != MFA_OK) return rr;
      const double rms = std::sqrt(res[0] / (double)npts);
      md->last_rms = rms;
      if (std::fabs(rms - rms_prev) <= tol_rms_stall * rms) {
        rc = MFA_OK;
        break;
      }
      rms_prev = rms;
    }
  }
  if (max_iters == 0) rc = MFA_OK;
  if (stall && status >= 0) {  // the residual decodes after the last read-back
    status = read_status(h);
    if (status < 0) rc = status;
  }
  if (rep) {
    rep->iters = md->iters;
    rep->status = rc;
    rep->dP_rel = md->last_dP;
    rep->jump_max = md->last_jump;
    if (stall && md->last_rms >= 0) {
      rep->rms_decoded = md->last_rms;
      rep->maxabs_decoded = res[1];
      rep->data_range = res[3] - res[2];
    }
  }
  return rc;
}

int mfa_decode(mfa_handle* h, const mfa_model* mdc, const double* pts, int64_t npts_q, const int32_t* deriv, void* out,
               int out_dtype, int out_on_device) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !out) return MFA_ERR_ARG;
  if (out_dtype != MFA_F32 && out_dtype != MFA_F64) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  int der[3] = {0, 0, 0};
  if (deriv)
    for (int a = 0; a < md->dim; ++a) {
      if (deriv[a] < 0 || deriv[a] > md->degree) return MFA_ERR_ARG;
      der[a] = deriv[a];
    }
  const size_t osz = out_dtype == MFA_F64 ? 8 : 4;
  if (pts) {
    if (npts_q < 0) return MFA_ERR_ARG;
    if (npts_q == 0) return MFA_OK;
    // scattered points: copy coordinates (host) to the workspace
    const size_t pbytes = (size_t)npts_q * md->dim * sizeof(double);
    const size_t obytes = out_on_device ? 0 : (size_t)npts_q * osz;
    // float-float models with clamped interfaces or NURBS weights decode from
    // an FP64 copy of their control points with the general basis kernel
    bool general = false;
    for (int a = 0; a < md->dim; ++a) general = general || md->axh[a].kmode != KMODE_FLOATING || !md->axh[a].wts.empty();
    const bool via64 = general && md->prec != MFA_PREC_FP64;
    const long long ncp = (long long)md->axh[0].n * md->axh[1].n * md->axh[2].n;
    const size_t cbytes = via64 ? (size_t)ncp * sizeof(double) : 0;
    int rc = ensure_ws(h, align256(pbytes) + align256(obytes) + align256(cbytes) + 256);
    if (rc != MFA_OK) return rc;
    double* dpts = (double*)h->ws;
    void* dout = out_on_device ? out : (void*)((char*)h->ws + align256(pbytes));
    double* P64 = (double*)((char*)h->ws + align256(pbytes) + align256(obytes));
    cudaError_t e = cudaMemcpyAsync(dpts, pts, pbytes, cudaMemcpyDefault, h->stream);
    if (via64) {
      TRACED(h, TR_MISC, (launch_cast<ff, double>((const ff*)md->P, P64, ncp, h->stream)));
      TRACED(h, TR_DECODE_POINTS,
             launch_decode_points<double>(md->L, md->lo, md->hi, dpts, npts_q, der, P64, dout, out_dtype, h->stream));
    } else if (md->prec == MFA_PREC_FP64)
      TRACED(h, TR_DECODE_POINTS,
             launch_decode_points<double>(md->L, md->lo, md->hi, dpts, npts_q, der, (const double*)md->P, dout,
                                          out_dtype, h->stream));
    else
      TRACED(h, TR_DECODE_POINTS,
             launch_decode_points<ff>(md->L, md->lo, md->hi, dpts, npts_q, der, (const ff*)md->P, dout, out_dtype,
                                      h->stream));
    if (e == cudaSuccess && !out_on_device)
      e = cudaMemcpyAsync(out, dout, (size_t)npts_q * osz, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    return cuda_status(e);
  }
  // full grid
  if (der[0] || der[1] || der[2]) return MFA_ERR_UNSUPPORTED;
  const long long n = (long long)md->axh[0].M * md->axh[1].M * md->axh[2].M;
  void* dst = out;
  void* tmp = nullptr;
  if (!out_on_device) {
    int rc = pool_alloc(h, &tmp, n * osz);
    if (rc != MFA_OK) return rc;
    dst = tmp;
  }
  int rc;
  if (md->prec == MFA_PREC_FP64)
    rc = out_dtype == MFA_F64 ? run_decode_grid<double, double, double>(md, (double*)dst, (const double*)nullptr)
                              : run_decode_grid<double, double, float>(md, (float*)dst, (const double*)nullptr);
  else
    rc = out_dtype == MFA_F64 ? run_decode_grid<ff, double, double>(md, (double*)dst, (const double*)nullptr)
                              : run_decode_grid<ff, double, float>(md, (float*)dst, (const double*)nullptr);
  cudaError_t e = cudaSuccess;
  if (rc == MFA_OK && !out_on_device) {
    e = cudaMemcpyAsync(out, dst, n * osz, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (tmp) pool_free(h, tmp);
  if (rc != MFA_OK) return rc;
  if (e == cudaSuccess) e = cudaGetLastError();
  return cuda_status(e);
}

int mfa_residual(mfa_handle* h, const mfa_model* mdc, const void* q, int q_dtype, int q_on_device, mfa_report* rep) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !rep) return MFA_ERR_ARG;
  if (!q) {  // the device copy this model staged from host data in mfa_encode
    if (!md->q_staged) return MFA_ERR_ARG;
    q = md->q_staged;
    q_dtype = md->q_staged_dtype;
    q_on_device = 1;
  }
  if (q_dtype != MFA_F32 && q_dtype != MFA_F64) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  const long long n = (long long)md->axh[0].M * md->axh[1].M * md->axh[2].M;
  const size_t qb = (size_t)n * (q_dtype == MFA_F64 ? 8 : 4);
  void* qtmp = nullptr;
  const void* qd = q;
  cudaError_t e = cudaSuccess;
  if (!q_on_device) {
    int rc = pool_alloc(h, &qtmp, qb);
    if (rc != MFA_OK) return rc;
    e = cudaMemcpyAsync(qtmp, q, qb, cudaMemcpyHostToDevice, h->stream);
    qd = qtmp;
  }
  double r[4] = {0, 0, 0, 0};
  int rc = e == cudaSuccess ? model_residual(md, qd, q_dtype, r) : cuda_status(e);
  if (qtmp) pool_free(h, qtmp);
  if (rc != MFA_OK) return rc;
  rep->rms_decoded = std::sqrt(r[0] / (double)n);
  rep->maxabs_decoded = r[1];
  rep->data_range = r[3] - r[2];
  rep->iters = md->iters;
  rep->dP_rel = md->last_dP;
  rep->jump_max = md->last_jump;
  int st = read_status(h);
  rep->status = st;
  return st < 0 ? st : MFA_OK;
}

int mfa_interface_jumps(mfa_handle* h, const mfa_model* mdc, int32_t max_order, mfa_report* rep) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !rep || md->batch || !md->has_state) return MFA_ERR_ARG;
  if (max_order < 0 || max_order > md->degree) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  const int R = max_order, p = md->degree, w = (R + 1) * (p + 1);
  // one-sided rows at every interface of every axis, then the neighbour pairs
  std::vector<double> rows;
  std::vector<int> rowcp;
  int row0[3] = {0, 0, 0};
  for (int a = 0; a < md->dim; ++a) {
    const AxisHost& ax = md->axh[a];
    row0[a] = (int)rowcp.size();
    for (int i = 0; i + 1 < ax.S; ++i)
      for (int side = 0; side < 2; ++side) {
        rows.resize(rows.size() + w);
        const int f = host_onesided_basis(ax, ax.subs[i].b, side, R, rows.data() + rows.size() - w);
        if (f < 0) return MFA_ERR_LAYOUT;
        rowcp.push_back(f);
      }
  }
  // samples along the other axes: the data points of the pair's common core
  auto core_pts = [&](int b, int piece, int& k0, int& k1) {
    const AxisHost& ax = md->axh[b];
    const AxisSub& sb = ax.subs[piece];
    if (ax.M == 1) {
      k0 = 0;
      k1 = 1;
      return;
    }
    const long long M1 = ax.M - 1;
    k0 = (int)((sb.a * M1 + ax.gspans - 1) / ax.gspans);
    k1 = (int)((sb.b * M1) / ax.gspans) + 1;
  };
  std::vector<JumpPair> pairs;
  const int S0 = md->axh[0].S, S1 = md->axh[1].S;
  for (int a = 0; a < md->dim; ++a)
    for (int sd = 0; sd < md->nsub; ++sd) {
      const int sa[3] = {sd % S0, (sd / S0) % S1, sd / (S0 * S1)};
      if (sa[a] + 1 >= md->axh[a].S) continue;
      JumpPair jp{};
      jp.s = sd;
      jp.t = sd + (a == 0 ? 1 : (a == 1 ? S0 : S0 * S1));
      jp.axis = a;
      jp.iface = row0[a] + 2 * sa[a];  // row of the left limit; the right limit follows it
      for (int b = 0; b < 3; ++b) {
        if (b == a) {
          jp.k0[b] = 0;
          jp.k1[b] = 1;
        } else {
          core_pts(b, sa[b], jp.k0[b], jp.k1[b]);
        }
      }
      pairs.push_back(jp);
    }
  for (int r = 0; r <= MFA_MAX_DEGREE; ++r) rep->jump_deriv[r] = 0.0;
  rep->jump_orders = R + 1;
  if (pairs.empty()) return MFA_OK;
  const size_t b_pairs = align256(pairs.size() * sizeof(JumpPair)), b_rows = align256(rows.size() * sizeof(double));
  const size_t b_cp = align256(rowcp.size() * sizeof(int));
  int rc = ensure_ws(h, b_pairs + b_rows + b_cp + 256);
  if (rc != MFA_OK) return rc;
  char* ws = (char*)h->ws;
  JumpPair* dpairs = (JumpPair*)ws;
  double* drows = (double*)(ws + b_pairs);
  int* dcp = (int*)(ws + b_pairs + b_rows);
  unsigned long long* dout = (unsigned long long*)(ws + b_pairs + b_rows + b_cp);
  cudaError_t e = cudaMemcpyAsync(dpairs, pairs.data(), pairs.size() * sizeof(JumpPair), cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dcp, rowcp.data(), rowcp.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, (R + 1) * sizeof(unsigned long long), h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  const int use_frames = md->iters > 0 ? 1 : 0;
  if (md->prec == MFA_PREC_FP64)
    TRACED(h, TR_MISC, launch_interface_jumps<double>(md->L, md->offL, (const double*)md->X,
                                                      (const double*)md->Pprev, use_frames, dpairs,
                                                      (int)pairs.size(), drows, dcp, R, dout, h->stream));
  else
    TRACED(h, TR_MISC, launch_interface_jumps<ff>(md->L, md->offL, (const ff*)md->X, (const ff*)md->Pprev, use_frames,
                                                  dpairs, (int)pairs.size(), drows, dcp, R, dout, h->stream));
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_pinned, dout, (R + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  std::memcpy(rep->jump_deriv, h->h_pinned, (R + 1) * sizeof(double));
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int64_t mfa_num_ctrl(const mfa_model* md) {
  if (!md) return MFA_ERR_ARG;
  return (int64_t)md->axh[0].n * md->axh[1].n * md->axh[2].n;
}

int mfa_get_ctrl(mfa_handle* h, const mfa_model* mdc, double* host_out, int64_t cap) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !host_out) return MFA_ERR_ARG;
  const long long n = mfa_num_ctrl(md);
  if (cap < n) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  int rc = ensure_ws(h, n * sizeof(double));
  if (rc != MFA_OK) return rc;
  if (md->prec == MFA_PREC_FP64)
    TRACED(h, TR_MISC, (launch_cast<double, double>((const double*)md->P, (double*)h->ws, n, h->stream)));
  else
    TRACED(h, TR_MISC, (launch_cast<ff, double>((const ff*)md->P, (double*)h->ws, n, h->stream)));
  cudaError_t e = cudaMemcpyAsync(host_out, h->ws, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int mfa_get_ctrl_async(mfa_handle* h, const mfa_model* mdc, double* host_out, int64_t cap) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !host_out) return MFA_ERR_ARG;
  const long long n = mfa_num_ctrl(md);
  if (cap < n) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  const size_t bytes = (size_t)n * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (h->rb_size < bytes) {
    // a larger staging buffer, once the last read out of the old one is done
    e = cudaEventSynchronize(h->rb_done);
    if (e != cudaSuccess) return cuda_status(e);
    pool_free(h, h->rb);
    h->rb = nullptr;
    h->rb_size = 0;
    const int rc = pool_alloc(h, &h->rb, bytes);
    if (rc != MFA_OK) return rc;
    h->rb_size = bytes;
  }
  // the cast waits for the previous read out of the buffer; the copy to the
  // host runs on the copy stream, beside whatever the handle's stream does next
  e = cudaStreamWaitEvent(h->stream, h->rb_done, 0);
  if (e != cudaSuccess) return cuda_status(e);
  if (md->prec == MFA_PREC_FP64)
    TRACED(h, TR_MISC, (launch_cast<double, double>((const double*)md->P, (double*)h->rb, n, h->stream)));
  else
    TRACED(h, TR_MISC, (launch_cast<ff, double>((const ff*)md->P, (double*)h->rb, n, h->stream)));
  e = cudaEventRecord(h->rb_ready, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->rb_ready, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, h->rb, bytes, cudaMemcpyDeviceToHost, h->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->rb_done, h->copy_stream);
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// Persistence: a fitted model to a file and back (layout, update rule,
// iteration count, global control points as stored on the device, and
// optionally the Schwarz state: B_L and the subdomain copies)
// ---------------------------------------------------------------------------

namespace {
constexpr char kMagic[8] = {'M', 'F', 'A', 'G', 'B', '3', 0, 1};
// version 2 adds the knot mode, NURBS weights and (with state) the lagged
// iterate; version 1 files (floating knots, no weights) are still read
constexpr int32_t kFileVersion = 2;

struct FileHeader {
  char magic[8];
  int32_t version, dim, degree, precision, update, flags, iters, knots;
  int64_t npts[3];
  int32_t nspans[3], nsub[3], overlap[3], wmask;  // wmask: bit a set when axis a has weights
  double lo[3], hi[3];
  double last_dP, last_jump;
  int64_t ncp, sizeL;
};
}  // namespace

int mfa_save(mfa_handle* h, const mfa_model* mdc, const char* path, int flags) {
  mfa_model* md = const_cast<mfa_model*>(mdc);
  if (!h || !md || md->h != h || !path || md->batch) return MFA_ERR_ARG;
  if ((flags & MFA_SAVE_STATE) && !md->has_state) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  FileHeader H{};
  std::memcpy(H.magic, kMagic, 8);
  H.version = kFileVersion;
  H.dim = md->dim;
  H.degree = md->degree;
  H.precision = md->prec;
  H.update = md->update == UPDATE_OWNER ? MFA_UPDATE_OWNER : MFA_UPDATE_AVERAGE;
  H.flags = flags & MFA_SAVE_STATE;
  H.iters = md->iters;
  H.knots = md->knots;
  for (int a = 0; a < 3; ++a) {
    if (!md->axh[a].wts.empty()) H.wmask |= 1 << a;
    H.npts[a] = md->axh[a].M;
    H.nspans[a] = md->axh[a].gspans;
    H.nsub[a] = md->axh[a].S;
    H.overlap[a] = md->overlap[a];
    H.lo[a] = md->lo[a];
    H.hi[a] = md->hi[a];
  }
  H.last_dP = md->last_dP;
  H.last_jump = md->last_jump;
  H.ncp = (long long)md->axh[0].n * md->axh[1].n * md->axh[2].n;
  H.sizeL = md->sizeL;
  const size_t es = elem_size(md->prec);
  const bool state = (flags & MFA_SAVE_STATE) != 0;
  std::vector<char> buf((size_t)H.ncp * es * (state ? 2 : 1) + (state ? 2 * (size_t)md->sizeL * es : 0));
  cudaError_t e = cudaMemcpyAsync(buf.data(), md->P, (size_t)H.ncp * es, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && state) {
    char* p2 = buf.data() + (size_t)H.ncp * es;
    e = cudaMemcpyAsync(p2, md->BL, (size_t)md->sizeL * es, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p2 + (size_t)md->sizeL * es, md->X, (size_t)md->sizeL * es, cudaMemcpyDeviceToHost,
                          h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p2 + 2 * (size_t)md->sizeL * es, md->Pprev, (size_t)H.ncp * es, cudaMemcpyDeviceToHost,
                          h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  FILE* f = std::fopen(path, "wb");
  if (!f) return MFA_ERR_IO;
  bool ok = std::fwrite(&H, sizeof(H), 1, f) == 1;
  for (int a = 0; a < md->dim && ok; ++a)
    for (const AxisSub& sb : md->axh[a].subs) {
      const int32_t c = sb.b - sb.a;
      ok = ok && std::fwrite(&c, sizeof(c), 1, f) == 1;
    }
  for (int a = 0; a < md->dim && ok; ++a)
    if (H.wmask & (1 << a))
      ok = std::fwrite(md->axh[a].wts.data(), sizeof(double), md->axh[a].wts.size(), f) == md->axh[a].wts.size();
  ok = ok && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MFA_OK : MFA_ERR_IO;
}

int mfa_load(mfa_handle* h, const char* path, mfa_model** out) {
  if (!h || !path || !out) return MFA_ERR_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return MFA_ERR_IO;
  FileHeader H{};
  bool ok = std::fread(&H, sizeof(H), 1, f) == 1 && std::memcmp(H.magic, kMagic, 8) == 0 &&
            (H.version == 1 || H.version == kFileVersion) && H.dim >= 1 && H.dim <= MFA_MAX_DIM &&
            H.degree >= 1 && H.degree <= MFA_MAX_DEGREE &&
            (H.precision == MFA_PREC_FP64 || H.precision == MFA_PREC_MIXED);
  if (ok && H.version == 1) {
    H.knots = MFA_KNOTS_FLOATING;
    H.wmask = 0;
  }
  ok = ok && (H.knots == MFA_KNOTS_FLOATING || H.knots == MFA_KNOTS_CLAMPED) && (H.wmask & ~7) == 0;
  std::vector<int32_t> cores[3];
  std::vector<double> wts[3];
  for (int a = 0; a < H.dim && ok; ++a) {
    ok = H.nsub[a] >= 1 && H.nsub[a] <= (1 << 20) && H.nspans[a] >= 1 && H.nspans[a] <= (1 << 30);
    if (ok) {
      cores[a].resize(H.nsub[a]);
      ok = std::fread(cores[a].data(), sizeof(int32_t), H.nsub[a], f) == (size_t)H.nsub[a];
    }
  }
  for (int a = 0; a < H.dim && ok; ++a)
    if (H.wmask & (1 << a)) {
      long long n = (long long)H.nspans[a] + H.degree;
      if (H.knots == MFA_KNOTS_CLAMPED && H.degree > 1) n += (long long)(H.degree - 1) * (H.nsub[a] - 1);
      wts[a].resize((size_t)n);
      ok = std::fread(wts[a].data(), sizeof(double), (size_t)n, f) == (size_t)n;
    }
  if (!ok) {
    std::fclose(f);
    return MFA_ERR_IO;
  }
  mfa_layout lay{};
  lay.dim = H.dim;
  lay.degree = H.degree;
  lay.precision = H.precision;
  lay.knots = H.knots;
  for (int a = 0; a < 3; ++a) {
    lay.weights[a] = wts[a].empty() ? nullptr : wts[a].data();
    lay.npts[a] = H.npts[a];
    lay.nspans[a] = H.nspans[a];
    lay.nsub[a] = H.nsub[a];
    lay.overlap[a] = H.overlap[a];
    lay.lo[a] = H.lo[a];
    lay.hi[a] = H.hi[a];
    lay.core_spans[a] = a < H.dim ? cores[a].data() : nullptr;
  }
  mfa_model* md = nullptr;
  size_t o_unused = 0;
  int rc = create_model(h, &lay, false, 0, &md, &o_unused);
  if (rc != MFA_OK) {
    std::fclose(f);
    return rc;
  }
  const size_t es = elem_size(md->prec);
  const long long ncp = (long long)md->axh[0].n * md->axh[1].n * md->axh[2].n;
  const bool state = (H.flags & MFA_SAVE_STATE) != 0;
  const bool has_prev = state && H.version >= 2;
  ok = H.ncp == ncp && (!state || H.sizeL == md->sizeL);
  std::vector<char> buf(ok ? (size_t)ncp * es * (has_prev ? 2 : 1) + (state ? 2 * (size_t)md->sizeL * es : 0) : 0);
  ok = ok && std::fread(buf.data(), 1, buf.size(), f) == buf.size();
  std::fclose(f);
  DeviceGuard g(h->device);
  cudaError_t e = cudaSuccess;
  if (ok) e = cudaMemcpyAsync(md->P, buf.data(), (size_t)ncp * es, cudaMemcpyHostToDevice, h->stream);
  if (ok && state && e == cudaSuccess) {
    const char* p2 = buf.data() + (size_t)ncp * es;
    e = cudaMemcpyAsync(md->BL, p2, (size_t)md->sizeL * es, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(md->X, p2 + (size_t)md->sizeL * es, (size_t)md->sizeL * es, cudaMemcpyHostToDevice,
                          h->stream);
    // the lagged iterate (the frames of the last step); a version-1 file has
    // none, and its P stands in for it
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(md->Pprev, has_prev ? p2 + 2 * (size_t)md->sizeL * es : buf.data(), (size_t)ncp * es,
                          cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (!ok || e != cudaSuccess) {
    pool_free(h, md->arena);
    pool_free(h, md->big);
    delete md;
    return ok ? cuda_status(e) : MFA_ERR_IO;
  }
  md->update = H.update == MFA_UPDATE_OWNER ? UPDATE_OWNER : UPDATE_AVERAGE;
  md->iters = H.iters;
  md->last_dP = H.last_dP;
  md->last_jump = H.last_jump;
  md->has_state = state;
  h->live_models++;
  *out = md;
  return MFA_OK;
}

int mfa_free(mfa_model* md) {
  if (!md) return MFA_ERR_ARG;
  mfa_handle* h = md->h;
  DeviceGuard g(h->device);
  pool_free(h, md->arena);
  pool_free(h, md->big);
  pool_free(h, md->tiles);
  h->live_models--;
  delete md;
  return MFA_OK;
}

int mfa_trace_enable(mfa_handle* h, int enable) {
  if (!h) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  trace_flush(h);
  if (enable && h->ev.empty()) {
    h->ev.resize(4096);
    for (auto& e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return MFA_ERR_CUDA;
  }
  h->trace_on = enable != 0;
  for (int i = 0; i < MFA_TRACE_CLASSES; ++i) {
    h->trace_ms[i] = 0.0;
    h->trace_n[i] = 0;
  }
  return MFA_OK;
}

int mfa_trace_read(mfa_handle* h, int32_t cls, double* total_ms, int64_t* launches) {
  if (!h || cls < 0 || cls >= MFA_TRACE_CLASSES) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  trace_flush(h);
  if (total_ms) *total_ms = h->trace_ms[cls];
  if (launches) *launches = h->trace_n[cls];
  return MFA_OK;
}

const char* mfa_trace_name(int32_t cls) {
  if (cls < 0 || cls >= MFA_TRACE_CLASSES) return "invalid";
  return kTraceNames[cls];
}

int mfa_sync(mfa_handle* h) {
  if (!h) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_stream);
  if (e != cudaSuccess) return cuda_status(e);
  return read_status(h);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent fits
// ---------------------------------------------------------------------------

struct mfa_batch {
  mfa_handle* h = nullptr;
  int count = 0;
  int prec = MFA_PREC_FP64;
  std::vector<mfa_instance> inst;
  std::vector<mfa_model*> groups;        // one per (dimension, degree)
  std::vector<long long> cp_off;         // [count + 1] control-point offsets, instance order
  std::vector<long long> q_len;          // values per instance
  long long q_total = 0;                 // length of the data array the instances span
  void* buf = nullptr;                   // control points of every instance (B_L, then solved in place)
  void* tab = nullptr;                   // device: q offsets [count], lengths [count]
  void* desc = nullptr;                  // device: InstDesc [count] for scattered decode
  void* staged = nullptr;                // device copy of host data
  int staged_dtype = MFA_F32;
  cudaGraphExec_t graph = nullptr;       // captured refit
  bool tuned = false;                    // tile sizes picked by timing (first refit)
  float tune_ms[9] = {};                 // fit time of every candidate (projection x solve block sizes)
  cudaStream_t cap = nullptr;            // private stream the refit is captured on
  const void* graph_q = nullptr;
  int graph_dtype = -1;
  // MFA_PREC_FP32: instance descriptors, projection and residual items, the
  // z-contraction tiles, the xy-reduced planes of 3-D instances, an FP32 copy
  // of the control points for the residual and the residual item totals
  void* b32 = nullptr;
  B32Inst* b32_inst = nullptr;
  B32Item* b32_pitems = nullptr;  // projection and residual items (instance by instance)
  int* b32_rfirst = nullptr;      // [2 count]: items of instance i are [rfirst[2 i], rfirst[2 i + 1])
  int* b32_ztile_inst = nullptr;
  long long* b32_ztile_base = nullptr;
  float* b32_R = nullptr;
  float* b32_Z = nullptr;         // y partial sums at warp boundaries of split 2-D instances
  float* b32_P32 = nullptr;
  double* b32_part = nullptr;
  int n_pitems = 0, n_ztiles = 0;
  // launches per class (0: 1-D and 2-D instances, 1: 3-D) and degree
  B32Caps caps[2][MFA_MAX_DEGREE + 1] = {};
  // iterative refinement of the instances whose FP32 error bound is large:
  // their projection items and z tiles, and the correction buffer (FP64)
  B32Item* b32_fitems = nullptr;
  int* b32_ftile_inst = nullptr;
  long long* b32_ftile_base = nullptr;
  ff* b32_dX = nullptr;
  int n_fitems = 0, n_ftiles = 0, n_refined = 0;
  // the decode's z expansion of 3-D instances (all of them, and the refined
  // ones) into DZ, laid out like R
  int* b32_etile_inst = nullptr;
  long long* b32_etile_base = nullptr;
  int* b32_fetile_inst = nullptr;
  long long* b32_fetile_base = nullptr;
  float* b32_DZ = nullptr;
  int n_etiles = 0, n_fetiles = 0;
  // the per-unit fit pipeline: unit u = class * (MFA_MAX_DEGREE + 1) +
  // degree; its z-contraction tiles (all, refined), refined z-expansion tiles
  // and control-point tiles (all, refined) are ranges [u_x[u], u_x[u + 1])
  // of the unit-sorted lists
  static constexpr int kUnits = 2 * (MFA_MAX_DEGREE + 1);
  int u_zt[kUnits + 1] = {}, u_ft[kUnits + 1] = {}, u_fe[kUnits + 1] = {}, u_ct[kUnits + 1] = {},
      u_rt[kUnits + 1] = {};
  long long* b32_ct_off = nullptr;
  int* b32_ct_len = nullptr;
  long long* b32_rt_off = nullptr;
  int* b32_rt_len = nullptr;
  // side streams on which the groups' independent work runs side by side
  // (forked from and joined back into the handle's stream; a captured refit
  // records them as parallel branches)
  cudaStream_t side[8] = {};
  int nside = 0;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int pfirst[2][MFA_MAX_DEGREE + 1] = {}, ffirst[2][MFA_MAX_DEGREE + 1] = {};
  int item_pts = 32768;  // data points per projection / residual item of a 3-D instance (autotuned)
};

namespace {

// Tile maps of a batch group for block sizes tc (projection), ts (solves) and
// te (decode): every operand of a launch split into blocks of that size, plus
// each instance's first tile of the last decode axis and its batch index.
// Replaces the group's previous maps.
int build_batch_tiles(mfa_handle* h, mfa_model* md, int tc, int ts, int te) {
  const std::vector<AxisOp>& ops = md->hops;
  const int ns = md->nsub, d = md->dim;
  std::vector<int> top;
  std::vector<long long> tbase;
  struct Span {
    TileMap* tm;
    size_t first;
  };
  std::vector<Span> spans;
  auto add = [&](TileMap* tm, int kind, int threads, bool fibres, int a) {
    spans.push_back({tm, top.size()});
    for (int t = 0; t < ns; ++t) {
      const View& v = ops[(size_t)kind * ns + t].out;
      const int a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;
      const long long n = fibres ? (long long)v.n[a1] * v.n[a2] : (long long)v.n[0] * v.n[1] * v.n[2];
      for (long long e = 0; e < n; e += threads) {
        top.push_back(t);
        tbase.push_back(e);
      }
    }
    tm->ntiles = (int)(top.size() - spans.back().first);
    tm->threads = threads;
  };
  for (int a = 0; a < d; ++a) {
    add(&md->tm_proj[a], OP_PROJ0 + a, tc, false, a);
    add(&md->tm_solve[a], OP_SOLVEL0 + a, ts, true, a);
    add(&md->tm_dec[a], OP_DEC0 + a, te, false, a);
  }
  std::vector<int> rfirst(ns + 1, 0), rid(ns);
  const size_t f0 = spans.back().first;  // the last span added is the last decode axis
  for (size_t k = f0; k < top.size(); ++k) rfirst[top[k] + 1]++;
  for (int t = 0; t < ns; ++t) {
    rfirst[t + 1] += rfirst[t];
    rid[t] = md->hmem[t];
  }
  // instances by decreasing size: the fused projection's CTA order
  std::vector<int> ord(ns);
  for (int t = 0; t < ns; ++t) ord[t] = t;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    const View& vx = ops[(size_t)OP_PROJ0 * ns + x].in;
    const View& vy = ops[(size_t)OP_PROJ0 * ns + y].in;
    return (long long)vx.n[0] * vx.n[1] * vx.n[2] > (long long)vy.n[0] * vy.n[1] * vy.n[2];
  });
  const size_t nt = top.size();
  void* mem = nullptr;
  int rc = pool_alloc(h, &mem, nt * (sizeof(int) + sizeof(long long)) + (3 * (size_t)ns + 1) * sizeof(int) + 16);
  if (rc != MFA_OK) return rc;
  long long* dbase = (long long*)mem;
  int* dop = (int*)(dbase + nt);
  int* dfirst = dop + nt;
  int* did = dfirst + ns + 1;
  int* dord = did + ns;
  cudaError_t e = cudaMemcpyAsync(dbase, tbase.data(), nt * sizeof(long long), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dop, top.data(), nt * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dfirst, rfirst.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(did, rid.data(), ns * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dord, ord.data(), ns * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    pool_free(h, mem);
    return cuda_status(e);
  }
  md->order = dord;
  pool_free(h, md->tiles);  // stream-ordered: after the launches that used the old maps
  md->tiles = mem;
  md->res_first = dfirst;
  md->res_id = did;
  for (const Span& sp : spans) {
    sp.tm->op = dop + sp.first;
    sp.tm->base = dbase + sp.first;
  }
  md->tile_c = tc;
  md->tile_s = ts;
  md->tile_e = te;
  return MFA_OK;
}

// One (dimension, degree) group as a model over virtual axes: axis a
// concatenates the group's instances, each a piece with its own knot vector;
// instance t of the group uses piece t on every axis of its dimension.
int build_batch_group(mfa_batch* b, int d, int p, const std::vector<int>& mem, mfa_model** out) {
  mfa_handle* h = b->h;
  mfa_model* md = new (std::nothrow) mfa_model();
  if (!md) return MFA_ERR_OOM;
  md->h = h;
  md->prec = b->prec;
  md->dim = d;
  md->degree = p;
  md->batch = true;
  md->use_fused = false;
  const int ns = (int)mem.size();
  for (int a = 0; a < 3; ++a) {
    AxisHost& ax = md->axh[a];
    if (a >= d) {
      int rc = build_axis(ax, 1, 1, 0, 1, nullptr, 0);
      if (rc != MFA_OK) {
        delete md;
        return rc;
      }
      continue;
    }
    ax = AxisHost{};
    ax.p = p;
    ax.S = ns;
    ax.pieces = 1;
    ax.M = 0;
    ax.n = 0;
    std::vector<int> ss;
    for (int t = 0; t < ns; ++t) {
      const mfa_instance& in = b->inst[mem[t]];
      AxisHost one;
      int rc = build_axis(one, in.npts[a], in.nspans[a], p, 1, nullptr, 0);
      if (rc != MFA_OK) {
        delete md;
        return rc;
      }
      AxisSub sb = one.subs[0];
      const int kbase = ax.M, cbase = ax.n;
      sb.k0 += kbase;
      sb.l0 += cbase;
      sb.bandL += cbase;
      sb.bandU += cbase;
      ax.subs.push_back(sb);
      // virtual spans share the control-point numbering: instance spans
      // [cbase, cbase + nspans), then p empty span numbers
      for (int j = 0; j < one.n; ++j) ss.push_back(kbase + (j < one.nspans ? one.span_start[j] : one.M));
      ax.M += one.M;
      ax.n += one.n;
    }
    ss.push_back(ax.M);
    ax.nspans = ax.n;
    ax.span_start = ss;
    ax.own_first.assign(ax.n, 0);
    ax.own_count.assign(ax.n, 1);
    ax.own_pick.assign(ax.n, 0);
    ax.own_tab.assign(ax.n, int4{0, 0, -1, 0});
    ax.nL_tab.resize(ns);
    ax.one_rng.assign(ns, int2{0, 0});
    for (int t = 0; t < ns; ++t) {
      const AxisSub& sb = ax.subs[t];
      ax.nL_tab[t] = sb.nL;
      ax.one_rng[t] = int2{sb.l0, sb.l0 + sb.nL};
      for (int l = 0; l < sb.nL; ++l) {
        ax.own_first[sb.l0 + l] = t;
        ax.own_tab[sb.l0 + l] = int4{t, l, -1, 0};
      }
    }
    ax.bandL_rows = ax.n;
    ax.bandU_rows = ax.n;
  }
  md->nsub = ns;
  // operand tables
  std::vector<AxisOp> ops((size_t)kOpKinds * ns, AxisOp{});
  std::vector<long long> offL(ns), offS1(ns), offS2(ns);
  long long a1 = 0, a2 = 0, d1 = 0, d2 = 0;
  for (int t = 0; t < ns; ++t) {
    const int i = mem[t];
    const mfa_instance& in = b->inst[i];
    AxisSub sb[3];
    int m[3], nL[3], sa[3];
    long long M[3];
    for (int a = 0; a < 3; ++a) {
      sa[a] = a < d ? t : 0;
      sb[a] = md->axh[a].subs[sa[a]];
      m[a] = sb[a].m;
      nL[a] = sb[a].nL;
      M[a] = a < d ? in.npts[a] : 1;
    }
    const long long szL = (long long)nL[0] * nL[1] * nL[2];
    offL[t] = b->cp_off[i];
    offS1[t] = a1;
    offS2[t] = a2;
    a1 += std::max((long long)nL[0] * m[1] * m[2], szL);
    a2 += std::max((long long)nL[0] * nL[1] * m[2], szL);
    md->sizeL += szL;
    for (int a = 0; a < 3; ++a) {
      md->maxm[a] = std::max(md->maxm[a], m[a]);
      md->maxnL[a] = std::max(md->maxnL[a], nL[a]);
      md->maxnU[a] = std::max(md->maxnU[a], nL[a]);
    }
    auto at = [&](int kind) -> AxisOp& { return ops[(size_t)kind * ns + t]; };
    // projection: instance grid -> S1 -> S2 -> its control points
    {
      View vin = make_view(in.q_offset, m[0], m[1], m[2], 1, M[0], M[0] * M[1]);
      int cur[3] = {m[0], m[1], m[2]};
      for (int a = 0; a < d; ++a) {
        cur[a] = nL[a];
        const long long off = (a == d - 1) ? offL[t] : (a == 0 ? offS1[t] : offS2[t]);
        View vout = contiguous(off, cur[0], cur[1], cur[2]);
        AxisOp& op = at(OP_PROJ0 + a);
        op.in = vin;
        op.out = vout;
        op.k0 = sb[a].k0;
        op.kend = sb[a].k0 + sb[a].m;
        op.c0 = sb[a].l0;
        op.sa = sa[a];
        md->maxOut[a] = std::max<long long>(md->maxOut[a], (long long)cur[0] * cur[1] * cur[2]);
        vin = vout;
      }
    }
    // solves in place over the control-point box
    for (int a = 0; a < 3; ++a) {
      AxisOp& opL = at(OP_SOLVEL0 + a);
      opL.out = contiguous(offL[t], nL[0], nL[1], nL[2]);
      opL.sa = sa[a];
      at(OP_SOLVEU0 + a) = opL;
      const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      md->maxFibL[a] = std::max(md->maxFibL[a], nL[o1] * nL[o2]);
      md->maxFibU[a] = md->maxFibL[a];
    }
    // decode: control points -> D1 -> D2 -> the instance grid of the output
    {
      int cur[3] = {nL[0], nL[1], nL[2]};
      View vin = contiguous(offL[t], cur[0], cur[1], cur[2]);
      for (int a = 0; a < d; ++a) {
        cur[a] = (int)M[a];
        const long long sz = (long long)cur[0] * cur[1] * cur[2];
        View vout;
        if (a == d - 1) {
          vout = make_view(in.q_offset, cur[0], cur[1], cur[2], 1, M[0], M[0] * M[1]);
        } else {
          long long& acc = (a == 0) ? d1 : d2;
          vout = contiguous(acc, cur[0], cur[1], cur[2]);
          acc += sz;
        }
        AxisOp& op = at(OP_DEC0 + a);
        op.in = vin;
        op.out = vout;
        op.k0 = sb[a].k0;
        op.kend = sb[a].k0 + sb[a].m;
        op.c0 = sb[a].l0;
        op.sa = sa[a];
        md->maxDec[a] = std::max(md->maxDec[a], sz);
        vin = vout;
      }
    }
  }
  md->sizeS1 = a1;
  md->sizeS2 = a2;
  md->decS1 = d1;
  md->decS2 = d2;
  size_t o_unused = 0;
  int rc = materialize_model(h, md, ops, offL, offS1, offS2, 0, &o_unused);
  if (rc != MFA_OK) {
    delete md;
    return rc;
  }
  md->BL = md->X = b->buf;
  md->P = b->buf;
  md->hops = ops;
  md->hmem = mem;
  md->L.diag = 1;
  // fused float-float kernels for 3-D groups run one CTA per instance
  // (largest first); they pay off only when no instance dominates: the
  // largest one, alone on an SM, must not outlast the group's work spread
  // over every CTA slot (2 per SM) by more than half.  Otherwise the tile
  // maps of the generic kernels spread each instance over many CTAs.  The
  // in-place stage-1 output needs >= 2 points per span on x.
  long long pmax = 0, ptot = 0;
  for (int t = 0; t < ns; ++t) {
    const View& v = ops[(size_t)OP_PROJ0 * ns + t].in;
    const long long np = (long long)v.n[0] * v.n[1] * v.n[2];
    pmax = std::max(pmax, np);
    ptot += np;
  }
  md->use_fused = (d == 3 && md->prec == MFA_PREC_MIXED && pmax * 2 * device_sm_count() <= 3 * ptot / 2);
  md->x_inplace_ok = true;
  for (const AxisSub& sb : md->axh[0].subs) {
    const long long Mi = sb.m, nsi = sb.w1 - sb.w0;
    long long prev = -1;
    for (long long k = 0; k < Mi && md->x_inplace_ok; ++k) {
      long long sk = Mi == 1 ? 0 : (k * nsi) / (Mi - 1);
      if (sk > nsi - 1) sk = nsi - 1;
      const long long cmax = sk - 1;
      if (cmax >= 0 && stage1_reach(cmax) > 4 * (k / 4) + 3) md->x_inplace_ok = false;
      if (k > 0 && sk - prev > 1) md->x_inplace_ok = false;  // one span per point at most
      prev = sk;
    }
  }
  rc = build_batch_tiles(h, md, kContractThreads, kSolveThreads, kExpandThreads);
  if (rc != MFA_OK) {
    md->BL = md->X = md->P = nullptr;
    pool_free(h, md->arena);
    pool_free(h, md->big);
    delete md;
    return rc;
  }
  h->live_models++;
  *out = md;
  return MFA_OK;
}

// Side streams of a batch (created on first use, one per group up to 8);
// 0 or 1 means the groups run on the handle's stream.
int batch_sides(mfa_batch* b) {
  const int want = std::min<int>(8, (int)b->groups.size());
  if (want <= 1) return 0;
  if (b->nside == 0) {
    if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    for (int i = 0; i < want; ++i) {
      if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      b->nside = i + 1;
    }
  }
  return b->nside;
}

// Every side stream waits for the work queued so far on the handle's stream.
void batch_fork(mfa_batch* b) {
  cudaEventRecord(b->fork_ev, b->h->stream);
  for (int i = 0; i < b->nside; ++i) cudaStreamWaitEvent(b->side[i], b->fork_ev, 0);
}

// The handle's stream waits for everything queued on the side streams.
void batch_join(mfa_batch* b) {
  for (int i = 0; i < b->nside; ++i) {
    cudaEventRecord(b->join_ev, b->side[i]);
    cudaStreamWaitEvent(b->h->stream, b->join_ev, 0);
  }
}

// The groups' fits (independent: own tables, own scratch, disjoint control
// points) run side by side, group g on side stream g mod nside.
template <typename T, typename TQ>
void batch_fit_all(mfa_batch* b, const TQ* q) {
  mfa_handle* h = b->h;
  const int ns = batch_sides(b);
  if (ns <= 1) {
    for (mfa_model* md : b->groups) run_encode<T, TQ>(md, q);
    return;
  }
  cudaStream_t main = h->stream;
  batch_fork(b);
  for (size_t g = 0; g < b->groups.size(); ++g) {
    h->stream = b->side[g % ns];  // run_encode launches on the handle's stream
    run_encode<T, TQ>(b->groups[g], q);
  }
  h->stream = main;
  batch_join(b);
}

template <typename T>
void batch_fit(mfa_batch* b, const void* q, int q_dtype) {
  if (q_dtype == MFA_F64)
    batch_fit_all<T, double>(b, (const double*)q);
  else
    batch_fit_all<T, float>(b, (const float*)q);
}

// FP32 data passes: the fused projection of every instance (one launch per
// class and degree), the z contraction of the 3-D instances, the banded
// solves of every group, and the FP32 copy of the control points the
// residual decodes from; then one refinement step for the instances whose
// FP32 error bound is large.
// One FP32 data pass over both classes: the launches of every (class,
// degree) side by side on the batch's side streams (disjoint outputs), so
// that no launch's tail idles the GPU.
void b32_pass(mfa_batch* b, int mode, const B32Item* items, int first[2][MFA_MAX_DEGREE + 1], const float* q,
              ff* X, double* part) {
  mfa_handle* h = b->h;
  const int ns = batch_sides(b);
  int k = 0;
  if (ns > 1) batch_fork(b);
  for (int c = 0; c < 2; ++c)
    launch_b32(mode, b->b32_inst, items, first[c], b->caps[c], q, b->b32_P32, b->b32_DZ, X, b->b32_R, b->b32_Z, part,
               h->stream, ns > 1 ? b->side : nullptr, ns > 1 ? ns : 0, &k);
  if (ns > 1) batch_join(b);
}

// The FP32 fit as one pipeline per (class, degree) unit, the units side by
// side on the batch's side streams: a unit's projection, z contraction,
// solves and FP32 copy, then its refinement step (z expansion, refinement
// projection, z contraction, solves, correction and FP32 copy), each unit in
// order on its own stream.  The units' instances, tiles and control points
// are disjoint, so one unit's latency-bound solves run beside other units'
// data passes.  The operations are those of the pass-by-pass order.
void batch_fit32_units(mfa_batch* b, const float* q) {
  mfa_handle* h = b->h;
  ff* X = (ff*)b->buf;
  const int ns = batch_sides(b);
  const long long ncp = b->cp_off[b->count];
  if (b->n_fitems) cudaMemsetAsync(b->b32_dX, 0, (size_t)ncp * sizeof(ff), h->stream);
  batch_fork(b);
  int k = 0;
  for (int c = 0; c < 2; ++c)
    for (int p = 1; p <= MFA_MAX_DEGREE; ++p) {
      if (b->pfirst[c][p] == b->pfirst[c][p - 1]) continue;
      const int u = c * (MFA_MAX_DEGREE + 1) + p;
      cudaStream_t st = b->side[k++ % ns];
      auto solves = [&](ff* x) {
        for (mfa_model* md : b->groups)
          if ((md->dim == 3) == (c == 1) && md->degree == p)
            for (int a = 0; a < md->dim; ++a)
              launch_band_solve<ff>(md->L, a, false, md->ops + (size_t)(OP_SOLVEL0 + a) * md->nsub, md->nsub,
                                    md->maxFibL[a], x, st, &md->tm_solve[a]);
      };
      launch_b32(B32_PROJECT, b->b32_inst, b->b32_pitems, b->pfirst[c], b->caps[c], q, nullptr, nullptr, X,
                 b->b32_R, b->b32_Z, nullptr, st, nullptr, 0, nullptr, p);
      launch_b32_zcontract(b->b32_inst, b->b32_ztile_inst + b->u_zt[u], b->b32_ztile_base + b->u_zt[u],
                           b->u_zt[u + 1] - b->u_zt[u], b->b32_R, X, st);
      solves(X);
      launch_b32_cast_tiles(b->b32_ct_off + b->u_ct[u], b->b32_ct_len + b->u_ct[u], b->u_ct[u + 1] - b->u_ct[u], X,
                            nullptr, b->b32_P32, st);
      if (b->ffirst[c][p] == b->ffirst[c][p - 1]) continue;
      launch_b32_zexpand(b->b32_inst, b->b32_fetile_inst + b->u_fe[u], b->b32_fetile_base + b->u_fe[u],
                         b->u_fe[u + 1] - b->u_fe[u], b->b32_P32, b->b32_DZ, st);
      launch_b32(B32_REFINE, b->b32_inst, b->b32_fitems, b->ffirst[c], b->caps[c], q, b->b32_P32, b->b32_DZ,
                 b->b32_dX, b->b32_R, b->b32_Z, nullptr, st, nullptr, 0, nullptr, p);
      launch_b32_zcontract(b->b32_inst, b->b32_ftile_inst + b->u_ft[u], b->b32_ftile_base + b->u_ft[u],
                           b->u_ft[u + 1] - b->u_ft[u], b->b32_R, b->b32_dX, st);
      solves(b->b32_dX);
      launch_b32_cast_tiles(b->b32_rt_off + b->u_rt[u], b->b32_rt_len + b->u_rt[u], b->u_rt[u + 1] - b->u_rt[u], X,
                            b->b32_dX, b->b32_P32, st);
    }
  batch_join(b);
}

void batch_fit32(mfa_batch* b, const float* q) {
  mfa_handle* h = b->h;
  // a traced fit runs pass by pass, so that each pass is timed on its own
  if (!h->trace_on && batch_sides(b) > 1) {
    batch_fit32_units(b, q);
    return;
  }
  ff* X = (ff*)b->buf;
  TRACED(h, TR_PROJECT_DATA, b32_pass(b, B32_PROJECT, b->b32_pitems, b->pfirst, q, X, nullptr));
  if (b->n_ztiles)
    TRACED(h, TR_PROJECT_REDUCED,
           launch_b32_zcontract(b->b32_inst, b->b32_ztile_inst, b->b32_ztile_base, b->n_ztiles, b->b32_R, X,
                                h->stream));
  // the groups' solves side by side (independent fibres of disjoint control points)
  auto solve_all = [&](ff* x) {
    const int ns = batch_sides(b);
    const int _ti = trace_begin(h);
    if (ns > 1) batch_fork(b);
    for (size_t g = 0; g < b->groups.size(); ++g) {
      mfa_model* md = b->groups[g];
      cudaStream_t st = ns > 1 ? b->side[g % ns] : h->stream;
      for (int a = 0; a < md->dim; ++a)
        launch_band_solve<ff>(md->L, a, false, md->ops + (size_t)(OP_SOLVEL0 + a) * md->nsub, md->nsub,
                              md->maxFibL[a], x, st, &md->tm_solve[a]);
    }
    if (ns > 1) batch_join(b);
    trace_end(h, TR_SOLVE_L, _ti);
  };
  solve_all(X);
  const long long ncp = b->cp_off[b->count];
  TRACED(h, TR_MISC, (launch_cast<ff, float>(X, b->b32_P32, ncp, h->stream)));
  if (b->n_fitems) {
    // one step of iterative refinement for the badly conditioned instances:
    // project r = q - N P32, solve, add the correction
    cudaMemsetAsync(b->b32_dX, 0, (size_t)ncp * sizeof(ff), h->stream);
    TRACED(h, TR_REFINE_DATA, {
      launch_b32_zexpand(b->b32_inst, b->b32_fetile_inst, b->b32_fetile_base, b->n_fetiles, b->b32_P32, b->b32_DZ,
                         h->stream);
      b32_pass(b, B32_REFINE, b->b32_fitems, b->ffirst, q, b->b32_dX, nullptr);
    });
    if (b->n_ftiles)
      TRACED(h, TR_PROJECT_REDUCED,
             launch_b32_zcontract(b->b32_inst, b->b32_ftile_inst, b->b32_ftile_base, b->n_ftiles, b->b32_R,
                                  b->b32_dX, h->stream));
    solve_all(b->b32_dX);
    TRACED(h, TR_MISC, launch_b32_add(X, b->b32_dX, ncp, h->stream));
    TRACED(h, TR_MISC, (launch_cast<ff, float>(X, b->b32_P32, ncp, h->stream)));
  }
}

void batch_fit_any(mfa_batch* b, const void* q, int q_dtype) {
  if (b->prec == MFA_PREC_FP32)
    batch_fit32(b, (const float*)q);
  else if (b->prec == MFA_PREC_FP64)
    batch_fit<double>(b, q, q_dtype);
  else
    batch_fit<ff>(b, q, q_dtype);
}

// Limits of the FP32 data-pass kernels for one instance: a row (padded to
// an odd pitch) fits one warp's staging buffer, the x basis values fit the
// CTA's table, and the open y control points of a streamed plane fit eight
// column groups.
bool b32_supported(const mfa_instance& in) {
  const int p = in.degree;
  const long long M0 = in.npts[0], n0 = (long long)in.nspans[0] + p;
  const int W = p < 4 ? 4 : 8;  // basis values per point in shared memory
  return (M0 | 1) <= kB32Stage && n0 <= kB32Threads && W * M0 <= 8192;
}

// Condition number of the normal matrix N^T N of one axis (M points
// u_k = k/(M-1), clamped uniform knots of nspans spans, degree p): the basis
// by the Cox-de Boor recurrence, the banded Gram matrix, its largest
// eigenvalue by power iteration and its smallest by inverse iteration
// (banded Cholesky solves).  An estimate, for choosing where the FP32 data
// passes need a refinement step.
double host_gram_cond(long long M, int ns, int p) {
  const int n = ns + p, w = p + 1;
  std::vector<double> A((size_t)n * w, 0.0);
  auto knot = [&](int i) { return (double)std::min(std::max(i - p, 0), ns) / ns; };
  double N[MFA_MAX_DEGREE + 1];
  for (long long k = 0; k < M; ++k) {
    const double u = M > 1 ? (double)k / (double)(M - 1) : 0.0;
    int j = M > 1 ? (int)((k * ns) / (M - 1)) : 0;
    j = std::min(j, ns - 1);
    const int i = j + p;
    N[0] = 1.0;
    for (int q = 1; q <= p; ++q) {
      double carry = 0.0;
      for (int r = 0; r < q; ++r) {
        const double tl = knot(i - q + r + 1), tr = knot(i + r + 1);
        const double wgt = N[r] / (tr - tl);
        const double right = (tr - u) * wgt, left = (u - tl) * wgt;
        N[r] = carry + right;
        carry = left;
      }
      N[q] = carry;
    }
    for (int r = 0; r <= p; ++r)
      for (int e = 0; r + e <= p; ++e) A[(size_t)(j + r) * w + e] += N[r] * N[r + e];
  }
  auto matvec = [&](const std::vector<double>& x, std::vector<double>& y) {
    std::fill(y.begin(), y.end(), 0.0);
    for (int r = 0; r < n; ++r)
      for (int e = 0; e <= p && r + e < n; ++e) {
        const double a = A[(size_t)r * w + e];
        y[r] += a * x[r + e];
        if (e) y[r + e] += a * x[r];
      }
  };
  // banded Cholesky A = L L^T, L(i, i-e) at F[i*w+e]
  std::vector<double> F((size_t)n * w, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int e = p; e >= 1; --e) {
      const int j = i - e;
      if (j < 0) continue;
      double sacc = A[(size_t)j * w + e];
      for (int f = e + 1; f <= p; ++f)
        if (i - f >= 0) sacc -= F[(size_t)i * w + f] * F[(size_t)j * w + (f - e)];
      F[(size_t)i * w + e] = sacc / F[(size_t)j * w];
    }
    double d = A[(size_t)i * w];
    for (int e = 1; e <= p; ++e)
      if (i - e >= 0) d -= F[(size_t)i * w + e] * F[(size_t)i * w + e];
    if (!(d > 0.0)) return 1e300;
    F[(size_t)i * w] = std::sqrt(d);
  }
  auto solve = [&](std::vector<double>& x) {
    for (int i = 0; i < n; ++i) {
      double v = x[i];
      for (int e = 1; e <= p && i - e >= 0; ++e) v -= F[(size_t)i * w + e] * x[i - e];
      x[i] = v / F[(size_t)i * w];
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = x[i];
      for (int e = 1; e <= p && i + e < n; ++e) v -= F[(size_t)(i + e) * w + e] * x[i + e];
      x[i] = v / F[(size_t)i * w];
    }
  };
  std::vector<double> x(n), y(n);
  auto normalise = [&](std::vector<double>& v) {
    double s2 = 0.0;
    for (double t : v) s2 += t * t;
    const double s = std::sqrt(s2);
    for (double& t : v) t /= s;
    return s;
  };
  for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.37 * ((i * 7919) % 13);
  normalise(x);
  double lmax = 0.0;
  for (int it = 0; it < 30; ++it) {
    matvec(x, y);
    lmax = normalise(y);
    x.swap(y);
  }
  for (int i = 0; i < n; ++i) x[i] = ((i * 7919) % 13) - 6.0 + 0.5;
  normalise(x);
  double inv = 0.0;
  for (int it = 0; it < 30; ++it) {
    solve(x);
    inv = normalise(x);
  }
  return lmax * inv;
}

// Device tables of the FP32 data passes: descriptors with each instance's
// chunk geometry, CTA items (3-D: ranges of planes of about item_pts points,
// split between eight warps; 2-D: the whole instance, split between warps by
// y knot spans; 1-D: the whole instance), each instance's item range, the
// launch capacities per class and degree, z-contraction tiles, and the
// subset of items and tiles that the refinement step reprojects.
int build_b32(mfa_batch* b) {
  mfa_handle* h = b->h;
  const int count = b->count;
  std::vector<B32Inst> D(count);
  long long rsize = 0;
  for (mfa_model* md : b->groups)
    for (int t = 0; t < md->nsub; ++t) {
      const int i = md->hmem[t];
      const mfa_instance& in = b->inst[i];
      B32Inst& d = D[i];
      d.dim = in.dim;
      d.p = in.degree;
      for (int a = 0; a < 3; ++a) {
        const bool act = a < in.dim;
        d.M[a] = act ? (int)in.npts[a] : 1;
        d.n[a] = act ? in.nspans[a] + in.degree : 1;
        d.kbase[a] = act ? md->axh[a].subs[t].k0 : 0;
        d.cbase[a] = act ? md->axh[a].subs[t].l0 : 0;
        d.span[a] = act ? md->L.ax[a].span : nullptr;
        d.vals[a] = act ? md->L.ax[a].vals_f : nullptr;
        d.sstart[a] = act ? md->L.ax[a].span_start : nullptr;
      }
      d.q_off = in.q_offset;
      d.x_off = b->cp_off[i];
      d.r_off = 0;
    }
  for (int i = 0; i < count; ++i)
    if (D[i].dim == 3) {
      D[i].r_off = rsize;
      rsize += (long long)D[i].M[2] * D[i].n[1] * D[i].n[0];
    }
  // chunk geometry of every instance and the launch capacities
  auto cls_of = [&](int i) { return D[i].dim == 3 ? 1 : 0; };
  B32Caps caps[2][MFA_MAX_DEGREE + 1];
  std::memset(caps, 0, sizeof(caps));
  for (int i = 0; i < count; ++i) {
    B32Inst& d = D[i];
    const int p = d.p, M0 = d.M[0], M1 = d.M[1], M2 = d.M[2], n0 = d.n[0], n1 = d.n[1];
    const int pitch = M0 | 1, n0s = n0 | 1, W = p < 4 ? 4 : 8;
    const int ns0 = n0 - p, ns1 = n1 - (d.dim >= 2 ? p : 0);
    int rows;
    if (d.dim == 1) {
      d.mode = 0;
      d.np = 1;
      rows = 1;
    } else if (M1 * pitch <= kB32Stage) {
      d.mode = 0;
      d.np = d.dim == 3 ? std::max(1, std::min(kB32Stage / (M1 * pitch), M2)) : 1;
      rows = d.np * M1;
    } else {
      d.mode = 1;
      d.np = 1;
      rows = std::min(kB32Stage / pitch, M1);
    }
    d.R = rows;
    // x segments: one lane per (pair of rows, segment) while row pairs alone
    // leave lanes idle
    const int pairs = (rows + 1) / 2;
    d.S = pairs >= 32 ? 1 : std::min(std::max(1, ns0 / p), std::max(1, 32 / pairs));
    B32Caps& c = caps[cls_of(i)][p];
    c.vb = std::max(c.vb, M0 * W);
    c.sx = std::max(c.sx, ns0 + 1);
    c.sy = std::max(c.sy, ns1 + 1);
    c.vy = std::max(c.vy, M1 * W);
    c.ysp = std::max(c.ysp, M1);
    c.stage = std::max(c.stage, rows * pitch);
    c.xr = std::max(c.xr, rows * n0s);
    if (d.mode == 1 && n0 > 32) c.ring = std::max(c.ring, (p + 1) * ((n0 + 31) / 32) * 32);
  }
  for (int k = 0; k < 2; ++k)
    for (int p = 1; p <= MFA_MAX_DEGREE; ++p)
      for (int mode : {B32_PROJECT, B32_REFINE, B32_RESIDUAL})
        if (b32_smem_bytes(caps[k][p], mode) > 220 * 1024) return MFA_ERR_UNSUPPORTED;
  // items by class and degree (one launch each), largest instances first,
  // the items of an instance contiguous
  std::vector<int> ord(count);
  for (int i = 0; i < count; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    if (cls_of(x) != cls_of(y)) return cls_of(x) < cls_of(y);
    if (D[x].p != D[y].p) return D[x].p < D[y].p;
    return b->q_len[x] > b->q_len[y];
  });
  const long long ipts = std::max(b->item_pts, 4096);
  std::vector<B32Item> pit;
  std::vector<int> rrange(2 * (size_t)count, 0);
  long long zsize = 0;
  for (int i : ord) {
    const B32Inst& d = D[i];
    rrange[2 * i] = (int)pit.size();
    if (d.dim == 3) {
      const long long plane = (long long)d.M[0] * d.M[1];
      const int unit = 8 * d.np;  // whole chunks for every warp
      int ppi = (int)std::min<long long>(d.M[2], ((ipts / plane + unit - 1) / unit) * unit);
      ppi = std::max(ppi, std::min(unit, d.M[2]));
      for (int k2 = 0; k2 < d.M[2]; k2 += ppi) {
        const int k2e = std::min(k2 + ppi, d.M[2]);
        pit.push_back(B32Item{i, k2 * d.M[1], k2e * d.M[1], std::min(8, k2e - k2), 0});
      }
    } else if (d.dim == 2) {
      const int ns1 = d.n[1] - d.p;
      const int nw = d.mode == 1 ? std::max(1, std::min(8, ns1 / d.p)) : 1;
      pit.push_back(B32Item{i, 0, d.M[1], nw, nw > 1 ? zsize : 0});
      if (nw > 1) zsize += 2LL * nw * d.p * d.n[0];
    } else {
      pit.push_back(B32Item{i, 0, 1, 1, 0});
    }
    rrange[2 * i + 1] = (int)pit.size();
  }
  // first[k][q]: items of class k and degree <= q end there (absolute)
  auto firsts = [&](const std::vector<B32Item>& v, int first[2][MFA_MAX_DEGREE + 1]) {
    int cnt[2][MFA_MAX_DEGREE + 1] = {};
    for (const B32Item& x : v) cnt[cls_of(x.inst)][D[x.inst].p]++;
    int acc = 0;
    for (int k = 0; k < 2; ++k)
      for (int q = 0; q <= MFA_MAX_DEGREE; ++q) {
        acc += cnt[k][q];
        first[k][q] = acc;
      }
  };
  firsts(pit, b->pfirst);
  // tile lists in (class, degree) unit order, so that every unit's tiles are
  // one range (the per-unit fit pipeline launches them unit by unit)
  auto unit_of = [&](int i) { return cls_of(i) * (MFA_MAX_DEGREE + 1) + D[i].p; };
  std::vector<int> uord(count);
  for (int i = 0; i < count; ++i) uord[i] = i;
  std::stable_sort(uord.begin(), uord.end(), [&](int x, int y) { return unit_of(x) < unit_of(y); });
  std::vector<int> zti, eti;
  std::vector<long long> ztb, etb;
  for (int i : uord)
    if (D[i].dim == 3) {
      // z contraction: kB32ZThreads (j1, j0) columns per tile
      const long long n = (long long)D[i].n[0] * D[i].n[1];
      for (long long e = 0; e < n; e += kB32ZThreads) {
        zti.push_back(i);
        ztb.push_back(e);
      }
      // z expansion for the decode: 256 values of DZ (M2 x n1 x n0) per tile
      const long long nz = (long long)D[i].M[2] * D[i].n[1] * D[i].n[0];
      for (long long e = 0; e < nz; e += 256) {
        eti.push_back(i);
        etb.push_back(e);
      }
    }
  // a refinement step where the FP32 error bound 2^-24 prod_a sqrt(cond(N_a^T N_a))
  // of the decoded values, relative to the data, exceeds 2e-6 (observed errors
  // stay below ~1.1x this bound; after one step they fall below 1e-6)
  // (condition numbers cached for the process: one estimate per axis shape)
  static std::mutex cond_mu;
  static std::map<std::tuple<long long, int, int>, double> conds;
  std::vector<char> refine(count, 0);
  for (int i = 0; i < count; ++i) {
    const mfa_instance& in = b->inst[i];
    double g = std::ldexp(1.0, -24);
    for (int a = 0; a < in.dim; ++a) {
      const auto key = std::make_tuple((long long)in.npts[a], in.nspans[a], in.degree);
      double c;
      {
        std::lock_guard<std::mutex> lk(cond_mu);
        auto itc = conds.find(key);
        c = itc == conds.end() ? -1.0 : itc->second;
      }
      if (c < 0.0) {
        c = host_gram_cond(in.npts[a], in.nspans[a], in.degree);
        std::lock_guard<std::mutex> lk(cond_mu);
        conds.emplace(key, c);
      }
      g *= std::sqrt(c);
    }
    refine[i] = g > 2e-6;
  }
  std::vector<B32Item> fit;
  for (const B32Item& x : pit)
    if (refine[x.inst]) fit.push_back(x);
  firsts(fit, b->ffirst);
  std::vector<int> fti, feti;
  std::vector<long long> ftb, fetb;
  for (size_t k = 0; k < zti.size(); ++k)
    if (refine[zti[k]]) {
      fti.push_back(zti[k]);
      ftb.push_back(ztb[k]);
    }
  for (size_t k = 0; k < eti.size(); ++k)
    if (refine[eti[k]]) {
      feti.push_back(eti[k]);
      fetb.push_back(etb[k]);
    }
  // control-point tiles of every instance and of the refined ones, unit by unit
  std::vector<long long> cto, rto;
  std::vector<int> ctl, rtl;
  constexpr int NU = mfa_batch::kUnits;
  int u_ct[NU + 1] = {}, u_rt[NU + 1] = {}, u_zt[NU + 1] = {}, u_ft[NU + 1] = {}, u_fe[NU + 1] = {};
  for (int i : uord) {
    const int u = unit_of(i);
    for (long long o = b->cp_off[i]; o < b->cp_off[i + 1]; o += kB32CastTile) {
      const int n = (int)std::min<long long>(kB32CastTile, b->cp_off[i + 1] - o);
      cto.push_back(o);
      ctl.push_back(n);
      u_ct[u + 1]++;
      if (refine[i]) {
        rto.push_back(o);
        rtl.push_back(n);
        u_rt[u + 1]++;
      }
    }
  }
  for (int t : zti) u_zt[unit_of(t) + 1]++;
  for (int t : fti) u_ft[unit_of(t) + 1]++;
  for (int t : feti) u_fe[unit_of(t) + 1]++;
  for (int u = 0; u < NU; ++u) {
    u_ct[u + 1] += u_ct[u];
    u_rt[u + 1] += u_rt[u];
    u_zt[u + 1] += u_zt[u];
    u_ft[u + 1] += u_ft[u];
    u_fe[u + 1] += u_fe[u];
  }
  int nref = 0;
  for (int i = 0; i < count; ++i) nref += refine[i];
  std::memcpy(b->caps, caps, sizeof(caps));
  Arena ar;
  const size_t o_inst = ar.take<B32Inst>(count), o_pit = ar.take<B32Item>(pit.size()),
               o_rf = ar.take<int>(2 * (size_t)count), o_zi = ar.take<int>(zti.size()),
               o_zb = ar.take<long long>(ztb.size()), o_fit = ar.take<B32Item>(fit.size()),
               o_fti = ar.take<int>(fti.size()), o_ftb = ar.take<long long>(ftb.size()),
               o_ei = ar.take<int>(eti.size()), o_eb = ar.take<long long>(etb.size()),
               o_fei = ar.take<int>(feti.size()), o_feb = ar.take<long long>(fetb.size()),
               o_cto = ar.take<long long>(cto.size()), o_ctl = ar.take<int>(ctl.size()),
               o_rto = ar.take<long long>(rto.size()), o_rtl = ar.take<int>(rtl.size());
  const size_t host_bytes = ar.used;
  const size_t o_R = ar.take<float>(rsize), o_Z = ar.take<float>(zsize), o_P = ar.take<float>(b->cp_off[count]),
               o_part = ar.take<double>(2 * pit.size()), o_dX = ar.take<ff>(nref ? b->cp_off[count] : 0),
               o_DZ = ar.take<float>(rsize);
  void* mem = nullptr;
  int rc = pool_alloc(h, &mem, ar.used);
  if (rc != MFA_OK) return rc;
  // the table image in the handle's pinned FP32 staging buffer, once its
  // previous upload has been read: the copy then needs no stream sync
  cudaEventSynchronize(h->stage32_done);
  if (h->h_stage32_cap < host_bytes) {
    if (h->h_stage32) cudaFreeHost(h->h_stage32);
    h->h_stage32 = nullptr;
    h->h_stage32_cap = 0;
    if (cudaMallocHost(&h->h_stage32, host_bytes) != cudaSuccess) {
      cudaGetLastError();
      h->h_stage32 = nullptr;
      pool_free(h, mem);
      return MFA_ERR_OOM;
    }
    h->h_stage32_cap = host_bytes;
  }
  char* const img = h->h_stage32;
  std::memcpy(img + o_inst, D.data(), sizeof(B32Inst) * D.size());
  std::memcpy(img + o_pit, pit.data(), sizeof(B32Item) * pit.size());
  std::memcpy(img + o_rf, rrange.data(), sizeof(int) * rrange.size());
  std::memcpy(img + o_zi, zti.data(), sizeof(int) * zti.size());
  std::memcpy(img + o_zb, ztb.data(), sizeof(long long) * ztb.size());
  std::memcpy(img + o_fit, fit.data(), sizeof(B32Item) * fit.size());
  std::memcpy(img + o_fti, fti.data(), sizeof(int) * fti.size());
  std::memcpy(img + o_ftb, ftb.data(), sizeof(long long) * ftb.size());
  std::memcpy(img + o_ei, eti.data(), sizeof(int) * eti.size());
  std::memcpy(img + o_eb, etb.data(), sizeof(long long) * etb.size());
  std::memcpy(img + o_fei, feti.data(), sizeof(int) * feti.size());
  std::memcpy(img + o_feb, fetb.data(), sizeof(long long) * fetb.size());
  std::memcpy(img + o_cto, cto.data(), sizeof(long long) * cto.size());
  std::memcpy(img + o_ctl, ctl.data(), sizeof(int) * ctl.size());
  std::memcpy(img + o_rto, rto.data(), sizeof(long long) * rto.size());
  std::memcpy(img + o_rtl, rtl.data(), sizeof(int) * rtl.size());
  cudaError_t e = cudaMemcpyAsync(mem, img, host_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(h->stage32_done, h->stream);
  if (e != cudaSuccess) {
    pool_free(h, mem);
    return cuda_status(e);
  }
  pool_free(h, b->b32);  // stream-ordered: after the launches that used the old tables
  b->b32 = mem;
  b->b32_inst = at_off<B32Inst>(mem, o_inst);
  b->b32_pitems = at_off<B32Item>(mem, o_pit);
  b->b32_rfirst = at_off<int>(mem, o_rf);
  b->b32_ztile_inst = at_off<int>(mem, o_zi);
  b->b32_ztile_base = at_off<long long>(mem, o_zb);
  b->b32_R = at_off<float>(mem, o_R);
  b->b32_Z = at_off<float>(mem, o_Z);
  b->b32_P32 = at_off<float>(mem, o_P);
  b->b32_part = at_off<double>(mem, o_part);
  b->b32_fitems = at_off<B32Item>(mem, o_fit);
  b->b32_ftile_inst = at_off<int>(mem, o_fti);
  b->b32_ftile_base = at_off<long long>(mem, o_ftb);
  b->b32_dX = nref ? at_off<ff>(mem, o_dX) : nullptr;
  b->b32_etile_inst = at_off<int>(mem, o_ei);
  b->b32_etile_base = at_off<long long>(mem, o_eb);
  b->b32_fetile_inst = at_off<int>(mem, o_fei);
  b->b32_fetile_base = at_off<long long>(mem, o_feb);
  b->b32_DZ = at_off<float>(mem, o_DZ);
  b->b32_ct_off = at_off<long long>(mem, o_cto);
  b->b32_ct_len = at_off<int>(mem, o_ctl);
  b->b32_rt_off = at_off<long long>(mem, o_rto);
  b->b32_rt_len = at_off<int>(mem, o_rtl);
  std::memcpy(b->u_ct, u_ct, sizeof(u_ct));
  std::memcpy(b->u_rt, u_rt, sizeof(u_rt));
  std::memcpy(b->u_zt, u_zt, sizeof(u_zt));
  std::memcpy(b->u_ft, u_ft, sizeof(u_ft));
  std::memcpy(b->u_fe, u_fe, sizeof(u_fe));
  b->n_pitems = (int)pit.size();
  b->n_ztiles = (int)zti.size();
  b->n_fitems = (int)fit.size();
  b->n_ftiles = (int)fti.size();
  b->n_etiles = (int)eti.size();
  b->n_fetiles = (int)feti.size();
  b->n_refined = nref;
  return MFA_OK;
}

// Grid decode of every group into out (instance layout of the data).
template <typename T, typename TOut>
int batch_decode_into(mfa_batch* b, TOut* out) {
  mfa_handle* h = b->h;
  size_t need = 0;
  for (mfa_model* md : b->groups) need = std::max<size_t>(need, (size_t)(md->decS1 + md->decS2) * sizeof(T));
  int rc = ensure_ws(h, std::max<size_t>(need, 256));
  if (rc != MFA_OK) return rc;
  for (mfa_model* md : b->groups) {
    T* s1 = (T*)h->ws;
    T* s2 = s1 + md->decS1;
    const int ns = md->nsub;
    const T* in = (const T*)md->X;
    for (int a = 0; a < md->dim; ++a) {
      const AxisOp* op = md->ops + (size_t)(OP_DEC0 + a) * ns;
      if (a == md->dim - 1) {
        TRACED(h, TR_DECODE_OUT,
               (launch_expand<T, TOut>(md->L, a, op, ns, md->maxDec[a], in, out, h->stream, &md->tm_dec[a])));
      } else {
        T* o = (a == 0) ? s1 : s2;
        TRACED(h, TR_DECODE_STAGE,
               (launch_expand<T, T>(md->L, a, op, ns, md->maxDec[a], in, o, h->stream, &md->tm_dec[a])));
        in = o;
      }
    }
  }
  return MFA_OK;
}

template <typename TOut>
int batch_decode_any(mfa_batch* b, TOut* out) {
  return f64_store(b->prec) ? batch_decode_into<double, TOut>(b, out) : batch_decode_into<ff, TOut>(b, out);
}

}  // namespace

namespace {
// Self-tuned tile sizes: the fit of every group (projection + solves) is timed
// on the stream for every pair of block sizes (projection 64 / 128 / 256,
// solves 32 / 64 / 128; one warm run, one timed run each) and the fastest
// pair is kept for every group.  The decode keeps 256.
// One group's fit (projection, iteration-0 solves) on the handle's stream.
void group_fit_any(mfa_batch* b, mfa_model* md, const void* q, int q_dtype) {
  if (b->prec == MFA_PREC_FP64) {
    if (q_dtype == MFA_F64)
      run_encode<double, double>(md, (const double*)q);
    else
      run_encode<double, float>(md, (const float*)q);
  } else {
    if (q_dtype == MFA_F64)
      run_encode<ff, double>(md, (const double*)q);
    else
      run_encode<ff, float>(md, (const float*)q);
  }
}

// The FP32 batch's float-float solves of one group.
void group_solve32(mfa_batch* b, mfa_model* md) {
  for (int a = 0; a < md->dim; ++a)
    launch_band_solve<ff>(md->L, a, false, md->ops + (size_t)(OP_SOLVEL0 + a) * md->nsub, md->nsub, md->maxFibL[a],
                          (ff*)b->buf, b->h->stream, &md->tm_solve[a]);
}

// Autotuning on the first refit, per (dimension, degree) group.
//  - FP64 / mixed: every group times its own fit for projection blocks of
//    64/128/256 threads x solve blocks of 32/64/128 (the elements a CTA
//    takes) and, for 3-D mixed groups, the fused one-CTA-per-instance path;
//    each group keeps its fastest candidate.
//  - FP32: the data passes' work per CTA item (3-D ranges of planes of about
//    16 K, 32 K or 128 K points), timed over the batch's projection, and
//    every group's solve block size, timed over that group's solves.
// The second of two runs of each candidate is kept.
int batch_autotune(mfa_batch* b, const void* q, int q_dtype) {
  mfa_handle* h = b->h;
  const int cand_c[3] = {64, 128, 256}, cand_s[3] = {32, 64, 128};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MFA_ERR_CUDA;
  const bool tr = h->trace_on;
  trace_flush(h);
  h->trace_on = false;
  int rc = MFA_OK;
  auto timed = [&](auto&& work) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == MFA_OK; ++rep) {
      cudaEventRecord(e0, h->stream);
      work();
      cudaEventRecord(e1, h->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = MFA_ERR_CUDA;
      cudaEventElapsedTime(&ms, e0, e1);
    }
    return ms;
  };
  for (mfa_model* md : b->groups)
    for (float& t : md->tune_ms) t = -1.f;
  for (float& t : b->tune_ms) t = 0.f;
  if (b->prec == MFA_PREC_FP32) {
    const int cand_items[3] = {16384, 32768, 131072};
    const float* qf = (const float*)q;
    float best = 1e30f;
    int bi = b->item_pts;
    for (int k = 0; k < 3 && rc == MFA_OK; ++k) {
      b->item_pts = cand_items[k];
      rc = build_b32(b);
      if (rc != MFA_OK) break;
      const float ms = timed([&] {
        for (int c = 0; c < 2; ++c)
          launch_b32(B32_PROJECT, b->b32_inst, b->b32_pitems, b->pfirst[c], b->caps[c], qf, nullptr, nullptr,
                     (ff*)b->buf, b->b32_R, b->b32_Z, nullptr, h->stream);
      });
      for (mfa_model* md : b->groups) md->tune_ms[3 + k] = ms;
      if (ms < best) {
        best = ms;
        bi = cand_items[k];
      }
    }
    if (rc == MFA_OK && b->item_pts != bi) {
      b->item_pts = bi;
      rc = build_b32(b);
    }
    for (int is = 0; is < 3 && rc == MFA_OK; ++is)
      for (mfa_model* md : b->groups) {
        rc = build_batch_tiles(h, md, md->tile_c, cand_s[is], kExpandThreads);
        if (rc != MFA_OK) break;
        md->tune_ms[is] = timed([&] { group_solve32(b, md); });
      }
    for (mfa_model* md : b->groups) {
      if (rc != MFA_OK) break;
      int bs = 0;
      for (int is = 1; is < 3; ++is)
        if (md->tune_ms[is] < md->tune_ms[bs]) bs = is;
      md->tune_best = md->tune_ms[bs];
      rc = build_batch_tiles(h, md, md->tile_c, cand_s[bs], kExpandThreads);
    }
  } else {
    // fused candidate first (3-D mixed groups), then the tiled grid
    std::vector<char> fused_ok(b->groups.size(), 0);
    for (size_t g = 0; g < b->groups.size() && rc == MFA_OK; ++g) {
      mfa_model* md = b->groups[g];
      if (md->dim != 3 || md->prec != MFA_PREC_MIXED) continue;
      const bool was = md->use_fused;
      md->use_fused = true;
      md->tune_ms[9] = timed([&] { group_fit_any(b, md, q, q_dtype); });
      fused_ok[g] = 1;
      md->use_fused = was;
    }
    for (int ic = 0; ic < 3 && rc == MFA_OK; ++ic)
      for (int is = 0; is < 3 && rc == MFA_OK; ++is)
        for (mfa_model* md : b->groups) {
          rc = build_batch_tiles(h, md, cand_c[ic], cand_s[is], kExpandThreads);
          if (rc != MFA_OK) break;
          const bool was = md->use_fused;
          md->use_fused = false;
          const float ms = timed([&] { group_fit_any(b, md, q, q_dtype); });
          md->use_fused = was;
          md->tune_ms[ic * 3 + is] = ms;
          b->tune_ms[ic * 3 + is] += ms;
        }
    for (size_t g = 0; g < b->groups.size() && rc == MFA_OK; ++g) {
      mfa_model* md = b->groups[g];
      int bk = 0;
      for (int k = 1; k < 9; ++k)
        if (md->tune_ms[k] < md->tune_ms[bk]) bk = k;
      const bool fz = fused_ok[g] && md->tune_ms[9] >= 0.f && md->tune_ms[9] < md->tune_ms[bk];
      md->use_fused = fz;
      md->tune_best = fz ? md->tune_ms[9] : md->tune_ms[bk];
      rc = build_batch_tiles(h, md, cand_c[bk / 3], cand_s[bk % 3], kExpandThreads);
    }
  }
  h->trace_on = tr;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == MFA_OK) b->tuned = true;
  return rc;
}
}  // namespace

int mfa_gram_condition(int64_t npts, int32_t nspans, int32_t degree, double* out) {
  if (!out || npts < 1 || nspans < 1 || degree < 1 || degree > MFA_MAX_DEGREE) return MFA_ERR_ARG;
  *out = host_gram_cond((long long)npts, nspans, degree);
  return MFA_OK;
}

int mfa_batch_info(const mfa_batch* b, mfa_batch_info_t* out) {
  if (!b || !out) return MFA_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->count = b->count;
  out->groups = (int32_t)b->groups.size();
  out->precision = b->prec;
  out->refined = b->n_refined;
  out->items = b->n_pitems;
  for (int i = 0; i < b->count; ++i) out->points += b->q_len[i];
  out->ctrl = b->cp_off[b->count];
  return MFA_OK;
}

int mfa_batch_group_tuning(const mfa_batch* b, int32_t group, mfa_group_tuning_t* out) {
  if (!b || !out || group < 0 || group >= (int)b->groups.size()) return MFA_ERR_ARG;
  const mfa_model* md = b->groups[group];
  std::memset(out, 0, sizeof(*out));
  out->dim = md->dim;
  out->degree = md->degree;
  out->instances = md->nsub;
  out->tile_c = md->tile_c;
  out->tile_s = md->tile_s;
  out->tile_e = md->tile_e;
  out->fused = md->dim == 3 && md->prec == MFA_PREC_MIXED && md->use_fused ? 1 : 0;
  out->item_pts = b->prec == MFA_PREC_FP32 ? b->item_pts : 0;
  out->chosen_ms = md->tune_best;
  for (int k = 0; k < MFA_TUNE_CANDIDATES; ++k) out->candidate_ms[k] = md->tune_ms[k];
  return b->tuned ? MFA_OK : MFA_NOT_CONVERGED;
}

int mfa_batch_tile_sizes(const mfa_batch* b, int32_t* sizes, float* candidate_ms) {
  if (!b || !sizes) return MFA_ERR_ARG;
  const mfa_model* md = b->groups.empty() ? nullptr : b->groups[0];
  sizes[0] = md ? md->tile_c : 0;
  sizes[1] = md ? md->tile_s : 0;
  sizes[2] = md ? md->tile_e : 0;
  if (candidate_ms)
    for (int i = 0; i < 9; ++i) candidate_ms[i] = b->tune_ms[i];
  return b->tuned ? MFA_OK : MFA_NOT_CONVERGED;
}

int mfa_encode_batch(mfa_handle* h, int32_t count, const mfa_instance* inst, const void* q, int q_dtype,
                     int q_on_device, int precision, mfa_batch** out) {
  if (!h || count < 1 || !inst || !q || !out) return MFA_ERR_ARG;
  *out = nullptr;
  if (q_dtype != MFA_F32 && q_dtype != MFA_F64) return MFA_ERR_ARG;
  if (precision != MFA_PREC_FP64 && precision != MFA_PREC_MIXED && precision != MFA_PREC_FP32) return MFA_ERR_ARG;
  if (precision == MFA_PREC_FP32) {
    // FP32 data passes read FP32 data, within the kernels' staging limits
    if (q_dtype != MFA_F32) return MFA_ERR_UNSUPPORTED;
    for (int i = 0; i < count; ++i)
      if (inst[i].dim >= 1 && inst[i].dim <= MFA_MAX_DIM && inst[i].degree >= 1 && !b32_supported(inst[i]))
        return MFA_ERR_UNSUPPORTED;
  }
  DeviceGuard g(h->device);
  mfa_batch* b = new (std::nothrow) mfa_batch();
  if (!b) return MFA_ERR_OOM;
  b->h = h;
  b->count = count;
  b->prec = precision;
  b->inst.assign(inst, inst + count);
  b->cp_off.assign(count + 1, 0);
  b->q_len.assign(count, 1);
  // validate, count control points, group by (dimension, degree)
  std::vector<std::vector<int>> grp((MFA_MAX_DIM + 1) * (MFA_MAX_DEGREE + 1));
  for (int i = 0; i < count; ++i) {
    const mfa_instance& in = b->inst[i];
    if (in.dim < 1 || in.dim > MFA_MAX_DIM || in.degree < 1 || in.degree > MFA_MAX_DEGREE || in.q_offset < 0) {
      delete b;
      return MFA_ERR_ARG;
    }
    long long ncp = 1, len = 1;
    for (int a = 0; a < in.dim; ++a) {
      if (in.npts[a] < 1 || in.npts[a] > (1LL << 30) || in.nspans[a] < 1) {
        delete b;
        return MFA_ERR_ARG;
      }
      ncp *= in.nspans[a] + in.degree;
      len *= in.npts[a];
    }
    b->cp_off[i + 1] = b->cp_off[i] + ncp;
    b->q_len[i] = len;
    b->q_total = std::max(b->q_total, in.q_offset + len);
    grp[in.dim * (MFA_MAX_DEGREE + 1) + in.degree].push_back(i);
  }
  const size_t es = elem_size(precision);
  const size_t qbytes = (size_t)b->q_total * (q_dtype == MFA_F64 ? 8 : 4);
  int rc = pool_alloc(h, &b->buf, (size_t)b->cp_off[count] * es);
  if (rc == MFA_OK) rc = pool_alloc(h, &b->tab, (size_t)count * 4 * sizeof(long long));
  if (rc == MFA_OK) rc = pool_alloc(h, &b->desc, (size_t)count * sizeof(InstDesc));
  if (rc == MFA_OK && !q_on_device) rc = pool_alloc(h, &b->staged, qbytes);
  if (rc != MFA_OK) {
    mfa_batch_free(b);
    return rc;
  }
  {
    std::vector<long long> t(2 * (size_t)count);
    for (int i = 0; i < count; ++i) {
      t[i] = b->inst[i].q_offset;
      t[count + i] = b->q_len[i];
    }
    std::vector<InstDesc> dd(count);
    for (int i = 0; i < count; ++i) {
      const mfa_instance& in = b->inst[i];
      InstDesc& D = dd[i];
      D.dim = in.dim;
      D.p = in.degree;
      for (int a = 0; a < 3; ++a) {
        D.nspans[a] = a < in.dim ? in.nspans[a] : 1;
        D.n[a] = a < in.dim ? in.nspans[a] + in.degree : 1;
      }
      D.cp_off = b->cp_off[i];
    }
    cudaError_t e = cudaMemcpyAsync(b->tab, t.data(), t.size() * sizeof(long long), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->desc, dd.data(), dd.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      mfa_batch_free(b);
      return cuda_status(e);
    }
  }
  for (int d = 1; d <= MFA_MAX_DIM; ++d)
    for (int p = 1; p <= MFA_MAX_DEGREE; ++p) {
      const std::vector<int>& mem = grp[d * (MFA_MAX_DEGREE + 1) + p];
      if (mem.empty()) continue;
      mfa_model* md = nullptr;
      rc = build_batch_group(b, d, p, mem, &md);
      if (rc != MFA_OK) {
        mfa_batch_free(b);
        return rc;
      }
      b->groups.push_back(md);
    }
  const void* qd = q;
  if (!q_on_device) {
    cudaError_t e = cudaMemcpyAsync(b->staged, q, qbytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      mfa_batch_free(b);
      return cuda_status(e);
    }
    qd = b->staged;
    b->staged_dtype = q_dtype;
  }
  if (precision == MFA_PREC_FP32) {
    rc = build_b32(b);
    if (rc != MFA_OK) {
      mfa_batch_free(b);
      return rc;
    }
  }
  batch_fit_any(b, qd, q_dtype);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    mfa_batch_free(b);
    return cuda_status(e);
  }
  int st = read_status(h);
  if (st < 0) {
    mfa_batch_free(b);
    return st;
  }
  *out = b;
  return MFA_OK;
}

int mfa_batch_refit(mfa_handle* h, mfa_batch* b, const void* q, int q_dtype) {
  if (!h || !b || b->h != h || !q) return MFA_ERR_ARG;
  if (q_dtype != MFA_F32 && q_dtype != MFA_F64) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  cudaError_t e = cudaSuccess;
  if (!b->tuned) {
    int rc = batch_autotune(b, q, q_dtype);
    if (rc != MFA_OK) return rc;
  }
  if (!b->graph || b->graph_q != q || b->graph_dtype != q_dtype) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    // capture the fit of every group once, on a private stream (the
    // handle's stream may be the legacy default stream, which cannot be
    // captured); tracing stays off inside the capture
    if (!b->cap) {
      e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        b->cap = nullptr;
        return cuda_status(e);
      }
    }
    const bool tr = h->trace_on;
    trace_flush(h);
    h->trace_on = false;
    cudaStream_t user = h->stream;
    h->stream = b->cap;
    cudaGraph_t gr = nullptr;
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      batch_fit_any(b, q, q_dtype);
      const cudaError_t e2 = cudaStreamEndCapture(b->cap, &gr);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = e2;
    }
    h->stream = user;
    h->trace_on = tr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return cuda_status(e);
    }
    b->graph_q = q;
    b->graph_dtype = q_dtype;
  }
  const int ti = trace_begin(h);
  e = cudaGraphLaunch(b->graph, h->stream);
  trace_end(h, TR_PROJECT_DATA, ti, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int64_t mfa_batch_num_ctrl(const mfa_batch* b) { return b ? (int64_t)b->cp_off[b->count] : (int64_t)MFA_ERR_ARG; }

int mfa_batch_ctrl_offsets(const mfa_batch* b, int64_t* host_off) {
  if (!b || !host_off) return MFA_ERR_ARG;
  for (int i = 0; i <= b->count; ++i) host_off[i] = b->cp_off[i];
  return MFA_OK;
}

int mfa_batch_get_ctrl(mfa_handle* h, const mfa_batch* b, double* host_out, int64_t cap) {
  if (!h || !b || b->h != h || !host_out) return MFA_ERR_ARG;
  const long long n = b->cp_off[b->count];
  if (cap < n) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  int rc = ensure_ws(h, (size_t)n * sizeof(double));
  if (rc != MFA_OK) return rc;
  if (f64_store(b->prec))
    TRACED(h, TR_MISC, (launch_cast<double, double>((const double*)b->buf, (double*)h->ws, n, h->stream)));
  else
    TRACED(h, TR_MISC, (launch_cast<ff, double>((const ff*)b->buf, (double*)h->ws, n, h->stream)));
  cudaError_t e = cudaMemcpyAsync(host_out, h->ws, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

namespace {
// Decoded error of every instance of every group: stage expansions into the
// workspace, then the last axis fused with E = Q - D over the tile map and a
// fixed-order per-instance reduction into out[2 * i], out[2 * i + 1].
template <typename T, typename TQ>
int batch_residual_into(mfa_batch* b, const TQ* q, double* out) {
  mfa_handle* h = b->h;
  // every group its own workspace region, so that the groups run side by side
  const size_t ng = b->groups.size();
  std::vector<size_t> woff(ng + 1, 0);
  for (size_t g = 0; g < ng; ++g) {
    const mfa_model* md = b->groups[g];
    const size_t sz = (size_t)(md->decS1 + md->decS2) * sizeof(T) +
                      2 * (size_t)md->tm_dec[md->dim - 1].ntiles * sizeof(double) + 64;
    woff[g + 1] = woff[g] + ((sz + 255) & ~(size_t)255);
  }
  int rc = ensure_ws(h, woff[ng]);
  if (rc != MFA_OK) return rc;
  const int nsd = batch_sides(b);
  cudaStream_t main = h->stream;
  if (nsd > 1) batch_fork(b);
  for (size_t g = 0; g < ng; ++g) {
    mfa_model* md = b->groups[g];
    if (nsd > 1) h->stream = b->side[g % nsd];
    T* s1 = (T*)((char*)h->ws + woff[g]);
    T* s2 = s1 + md->decS1;
    double* tpart = (double*)(((uintptr_t)(s2 + md->decS2) + 15) & ~(uintptr_t)15);
    const int ns = md->nsub, d = md->dim;
    const T* in = (const T*)md->X;
    for (int a = 0; a < d - 1; ++a) {
      const AxisOp* op = md->ops + (size_t)(OP_DEC0 + a) * ns;
      T* o = (a == 0) ? s1 : s2;
      TRACED(h, TR_DECODE_STAGE,
             (launch_expand<T, T>(md->L, a, op, ns, md->maxDec[a], in, o, h->stream, &md->tm_dec[a])));
      in = o;
    }
    const AxisOp* op = md->ops + (size_t)(OP_DEC0 + d - 1) * ns;
    TRACED_N(h, TR_RESIDUAL, 2,
             (launch_expand_residual_tiles<T, TQ>(md->L, d - 1, op, in, q, md->tm_dec[d - 1], tpart, md->res_first,
                                                  md->res_id, ns, out, h->stream)));
  }
  h->stream = main;
  if (nsd > 1) batch_join(b);
  return MFA_OK;
}
}  // namespace

int mfa_batch_residual(mfa_handle* h, const mfa_batch* bc, const void* q, int q_dtype, int q_on_device, double* rms,
                       double* maxabs) {
  mfa_batch* b = const_cast<mfa_batch*>(bc);
  if (!h || !b || b->h != h || !rms || !maxabs) return MFA_ERR_ARG;
  if (!q) {
    if (!b->staged) return MFA_ERR_ARG;
    q = b->staged;
    q_dtype = b->staged_dtype;
    q_on_device = 1;
  }
  if (q_dtype != MFA_F32 && q_dtype != MFA_F64) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  const size_t qb = (size_t)b->q_total * (q_dtype == MFA_F64 ? 8 : 4);
  void* qtmp = nullptr;
  void* res = nullptr;
  cudaError_t e = cudaSuccess;
  int rc = pool_alloc(h, &res, 2 * (size_t)b->count * sizeof(double));
  if (rc == MFA_OK && !q_on_device) {
    rc = pool_alloc(h, &qtmp, qb);
    if (rc == MFA_OK) e = cudaMemcpyAsync(qtmp, q, qb, cudaMemcpyHostToDevice, h->stream);
    q = qtmp;
  }
  if (rc == MFA_OK && e == cudaSuccess && b->prec == MFA_PREC_FP32 && q_dtype != MFA_F32) rc = MFA_ERR_UNSUPPORTED;
  if (rc == MFA_OK && e == cudaSuccess) {
    if (b->prec == MFA_PREC_FP32) {
      TRACED(h, TR_RESIDUAL, {
        launch_b32_zexpand(b->b32_inst, b->b32_etile_inst, b->b32_etile_base, b->n_etiles, b->b32_P32, b->b32_DZ,
                           h->stream);
        b32_pass(b, B32_RESIDUAL, b->b32_pitems, b->pfirst, (const float*)q, nullptr, b->b32_part);
      });
      TRACED(h, TR_REDUCE, launch_b32_reduce(b->b32_rfirst, b->count, b->b32_part, (double*)res, h->stream));
    } else if (b->prec == MFA_PREC_FP64)
      rc = q_dtype == MFA_F64 ? batch_residual_into<double, double>(b, (const double*)q, (double*)res)
                              : batch_residual_into<double, float>(b, (const float*)q, (double*)res);
    else
      rc = q_dtype == MFA_F64 ? batch_residual_into<ff, double>(b, (const double*)q, (double*)res)
                              : batch_residual_into<ff, float>(b, (const float*)q, (double*)res);
  }
  std::vector<double> hr(2 * (size_t)b->count);
  if (rc == MFA_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(hr.data(), res, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (qtmp) pool_free(h, qtmp);
  if (res) pool_free(h, res);
  if (rc != MFA_OK) return rc;
  if (e != cudaSuccess) return cuda_status(e);
  for (int i = 0; i < b->count; ++i) {
    rms[i] = std::sqrt(hr[2 * i] / (double)b->q_len[i]);
    maxabs[i] = hr[2 * i + 1];
  }
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int mfa_batch_decode(mfa_handle* h, const mfa_batch* bc, void* out, int out_dtype, int out_on_device) {
  mfa_batch* b = const_cast<mfa_batch*>(bc);
  if (!h || !b || b->h != h || !out) return MFA_ERR_ARG;
  if (out_dtype != MFA_F32 && out_dtype != MFA_F64) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  const size_t osz = out_dtype == MFA_F64 ? 8 : 4;
  void* dst = out;
  int rc = MFA_OK;
  if (!out_on_device) rc = pool_alloc(h, &dst, (size_t)b->q_total * osz);
  if (rc != MFA_OK) return rc;
  rc = out_dtype == MFA_F64 ? batch_decode_any<double>(b, (double*)dst) : batch_decode_any<float>(b, (float*)dst);
  cudaError_t e = cudaSuccess;
  if (rc == MFA_OK && !out_on_device)
    e = cudaMemcpyAsync(out, dst, (size_t)b->q_total * osz, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (!out_on_device) pool_free(h, dst);
  if (rc != MFA_OK) return rc;
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

int mfa_batch_free(mfa_batch* b) {
  if (!b) return MFA_ERR_ARG;
  mfa_handle* h = b->h;
  DeviceGuard g(h->device);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->nside) cudaStreamSynchronize(h->stream);
  for (int i = 0; i < b->nside; ++i) cudaStreamDestroy(b->side[i]);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (b->join_ev) cudaEventDestroy(b->join_ev);
  for (mfa_model* md : b->groups) {
    md->BL = md->X = md->P = nullptr;
    mfa_free(md);
  }
  pool_free(h, b->buf);
  pool_free(h, b->tab);
  pool_free(h, b->desc);
  pool_free(h, b->staged);
  pool_free(h, b->b32);
  delete b;
  return MFA_OK;
}

namespace mfa {
// Scattered decode of batch instances on any handle h (the batch's device
// tables are only read); host or device arrays.
int batch_decode_points_impl(mfa_handle* h, const mfa_batch* b, int32_t nq, const int32_t* qinst,
                             const int64_t* pt_off, const double* pts, double* out, int on_device) {
  if (!h || !b || nq < 1 || !qinst || !pt_off || !pts || !out) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  long long npts = 0;
  const int32_t* dq = qinst;
  const long long* doff = (const long long*)pt_off;
  const double* dp = pts;
  double* dout = out;
  void* tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    if (pt_off[0] != 0) return MFA_ERR_ARG;
    for (int k = 0; k < nq; ++k) {
      if (qinst[k] < 0 || qinst[k] >= b->count || pt_off[k + 1] < pt_off[k]) return MFA_ERR_ARG;
    }
    npts = pt_off[nq];
    const size_t bytes = (size_t)nq * sizeof(int32_t) + (size_t)(nq + 1) * sizeof(long long) +
                         (size_t)npts * 3 * sizeof(double) + (size_t)npts * sizeof(double) + 64;
    int rc = pool_alloc(h, &tmp, bytes);
    if (rc != MFA_OK) return rc;
    char* c = (char*)tmp;
    long long* o = (long long*)c;
    double* pp = (double*)(o + nq + 1);
    double* ov = pp + 3 * npts;
    int32_t* qi = (int32_t*)(ov + npts);
    e = cudaMemcpyAsync(o, pt_off, (size_t)(nq + 1) * sizeof(long long), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(qi, qinst, (size_t)nq * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && npts)
      e = cudaMemcpyAsync(pp, pts, (size_t)npts * 3 * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    dq = qi;
    doff = o;
    dp = pp;
    dout = ov;
  } else {
    // the point count is needed for the grid: read the last offset
    e = cudaMemcpyAsync(h->h_pinned, pt_off + nq, sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) std::memcpy(&npts, h->h_pinned, sizeof(long long));
  }
  if (e == cudaSuccess && npts > 0) {
    int p_uniform = b->inst.empty() ? 0 : b->inst[0].degree;
    for (const mfa_instance& in : b->inst)
      if (in.degree != p_uniform) p_uniform = 0;
    if (f64_store(b->prec))
      TRACED(h, TR_DECODE_POINTS, (launch_decode_points_inst<double>((const InstDesc*)b->desc, dq, doff, nq, npts, dp,
                                                                     (const double*)b->buf, dout, p_uniform,
                                                                     h->stream)));
    else
      TRACED(h, TR_DECODE_POINTS, (launch_decode_points_inst<ff>((const InstDesc*)b->desc, dq, doff, nq, npts, dp,
                                                                 (const ff*)b->buf, dout, p_uniform, h->stream)));
  }
  if (e == cudaSuccess && !on_device && npts > 0)
    e = cudaMemcpyAsync(out, dout, (size_t)npts * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (tmp) pool_free(h, tmp);
  if (e != cudaSuccess) return cuda_status(e);
  int st = read_status(h);
  return st < 0 ? st : MFA_OK;
}

// Control points of one instance as FP64 into host memory, on handle h.
int batch_instance_ctrl(mfa_handle* h, const mfa_batch* b, int index, double* host_out, int64_t cap) {
  if (!h || !b || index < 0 || index >= b->count || !host_out) return MFA_ERR_ARG;
  const long long n = b->cp_off[index + 1] - b->cp_off[index];
  if (cap < n) return MFA_ERR_ARG;
  DeviceGuard g(h->device);
  int rc = ensure_ws(h, (size_t)n * sizeof(double));
  if (rc != MFA_OK) return rc;
  if (f64_store(b->prec))
    launch_cast<double, double>((const double*)b->buf + b->cp_off[index], (double*)h->ws, n, h->stream);
  else
    launch_cast<ff, double>((const ff*)b->buf + b->cp_off[index], (double*)h->ws, n, h->stream);
  cudaError_t e = cudaMemcpyAsync(host_out, h->ws, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? MFA_OK : cuda_status(e);
}

long long batch_instance_num_ctrl(const mfa_batch* b, int index) { return b->cp_off[index + 1] - b->cp_off[index]; }
}  // namespace mfa

int mfa_batch_decode_points(mfa_handle* h, const mfa_batch* b, int32_t nq, const int32_t* qinst,
                            const int64_t* pt_off, const double* pts, double* out, int on_device) {
  if (!h || !b || b->h != h) return MFA_ERR_ARG;
  return mfa::batch_decode_points_impl(h, b, nq, qinst, pt_off, pts, out, on_device);
}

