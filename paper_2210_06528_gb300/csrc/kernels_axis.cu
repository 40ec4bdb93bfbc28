// Batched one-axis tensor operations over every subdomain at once.
// Every launch covers all subdomains: blockIdx.y selects the subdomain, the x
// dimension covers its output elements.  The per-subdomain operand views are
// built once on the host (AxisOp tables) and kept on the device.
#include <algorithm>

#include "mfa_internal.cuh"

namespace mfa {

template <typename T>
__device__ __forceinline__ const T* basis_vals(const AxisDev& ax);
template <>
__device__ __forceinline__ const double* basis_vals<double>(const AxisDev& ax) { return ax.vals_d; }
template <>
__device__ __forceinline__ const float* basis_vals<float>(const AxisDev& ax) { return ax.vals_f; }
template <>
__device__ __forceinline__ const ff* basis_vals<ff>(const AxisDev& ax) { return ax.vals_ff; }

template <typename T>
__device__ __forceinline__ const T* fac_L(const AxisDev& ax);
template <>
__device__ __forceinline__ const double* fac_L<double>(const AxisDev& ax) { return ax.facL_d; }
template <>
__device__ __forceinline__ const float* fac_L<float>(const AxisDev& ax) { return ax.facL_f; }
template <>
__device__ __forceinline__ const ff* fac_L<ff>(const AxisDev& ax) { return ax.facL_ff; }
template <typename T>
__device__ __forceinline__ const T* fac_U(const AxisDev& ax);
template <>
__device__ __forceinline__ const double* fac_U<double>(const AxisDev& ax) { return ax.facU_d; }
template <>
__device__ __forceinline__ const float* fac_U<float>(const AxisDev& ax) { return ax.facU_f; }
template <>
__device__ __forceinline__ const ff* fac_U<ff>(const AxisDev& ax) { return ax.facU_ff; }

// Operand and element of this thread: from the tile map when there is one,
// else operand blockIdx.y and element blockIdx.x * blockDim.x + threadIdx.x.
__device__ __forceinline__ void tile_of(const TileMap& tm, int& opi, long long& idx) {
  if (tm.op) {
    opi = tm.op[blockIdx.x];
    idx = tm.base[blockIdx.x] + threadIdx.x;
  } else {
    opi = blockIdx.y;
    idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  }
}

// The operand of this block, copied once into shared memory: every thread of
// a block works on the same operand, so the descriptor is read once per
// block instead of once per thread.  Called by all threads (it has a barrier).
__device__ __forceinline__ const AxisOp& block_op(const AxisOp* ops, int opi) {
  __shared__ AxisOp sop;
  static_assert(sizeof(AxisOp) % sizeof(int) == 0, "AxisOp is copied as ints");
  constexpr int nw = (int)(sizeof(AxisOp) / sizeof(int));
  for (int i = threadIdx.x; i < nw; i += blockDim.x)
    reinterpret_cast<int*>(&sop)[i] = reinterpret_cast<const int*>(ops + opi)[i];
  __syncthreads();
  return sop;
}

__device__ __forceinline__ void unflatten(long long idx, const int* n, int* o) {
  if (idx < (1LL << 31)) {  // 32-bit unsigned division is several times cheaper
    const unsigned i = (unsigned)idx, n0 = (unsigned)n[0], n1 = (unsigned)n[1];
    const unsigned r = i / n0;
    o[0] = (int)(i - r * n0);
    const unsigned r2 = r / n1;
    o[1] = (int)(r - r2 * n1);
    o[2] = (int)r2;
    return;
  }
  o[0] = (int)(idx % n[0]);
  long long r = idx / n[0];
  o[1] = (int)(r % n[1]);
  o[2] = (int)(r / n[1]);
}

__device__ __forceinline__ bool finite_val(float x) { return isfinite(x); }
__device__ __forceinline__ bool finite_val(double x) { return isfinite(x); }
__device__ __forceinline__ bool finite_val(ff x) { return isfinite(x.hi); }

// Projection along one axis: out[l] = sum_k N_{c0+l}(u_{k}) in[k - k0] over
// the points k of the window that lie in the support of control point c0+l,
// i.e. whose span is in [c0+l-p, c0+l] (the N^T Q assembly of the normal
// equations, Eq. minimization-problem).  When reading raw data the kernel also
// flags non-finite input.
template <typename T, typename TIn, int AXIS>
__global__ void k_contract(LayoutDev L, const AxisOp* ops, const TIn* __restrict__ in,
                           T* __restrict__ out, int* status, TileMap tm) {
  constexpr int axis = AXIS;
  int opi;
  long long idx;
  tile_of(tm, opi, idx);
  const AxisOp& op = block_op(ops, opi);
  const long long nout = (long long)op.out.n[0] * op.out.n[1] * op.out.n[2];
  if (idx >= nout) return;
  int o[3];
  unflatten(idx, op.out.n, o);
  const AxisDev& ax = L.ax[axis];
  const int p = ax.p, w = p + 1;
  const int g = op.c0 + o[axis];
  int lo = g - p < 0 ? 0 : g - p;
  int hi = g + 1 > ax.nspans ? ax.nspans : g + 1;
  int kb = ax.span_start[lo], ke = ax.span_start[hi];
  if (kb < op.k0) kb = op.k0;
  if (ke > op.kend) ke = op.kend;
  long long base = op.in.off;
  for (int a = 0; a < 3; ++a)
    if (a != axis) base += (long long)o[a] * op.in.st[a];
  const long long sk = op.in.st[axis];
  const T* v = basis_vals<T>(ax);
  T acc = 0;
  bool bad = false;
  for (int k = kb; k < ke; ++k) {
    const TIn x = in[base + (long long)(k - op.k0) * sk];
    bad |= !finite_val(x);
    acc += v[(long long)k * w + (g - ax.span[k])] * (T)x;
  }
  if (bad && status) atomicExch(status, MFA_ERR_NONFINITE);
  const View& ov = op.out;
  out[ov.off + o[0] * ov.st[0] + o[1] * ov.st[1] + o[2] * ov.st[2]] = acc;
}

// Decode along one axis: out[k] = sum_r N_{span(k)+r}(u_k) in[span(k)+r-c0],
// terms whose control point lies outside the input range are zero (R P,
// Algorithm 1 error step).
template <typename T, int axis>
__device__ __forceinline__ T expand_one(const AxisDev& ax, const AxisOp& op, const int* o,
                                        const T* __restrict__ in) {
  const int p = ax.p, w = p + 1;
  const int k = op.k0 + o[axis];
  const int j = ax.span[k];
  long long base = op.in.off;
  for (int a = 0; a < 3; ++a)
    if (a != axis) base += (long long)o[a] * op.in.st[a];
  const long long sc = op.in.st[axis];
  const T* v = basis_vals<T>(ax) + (long long)k * w;
  T acc = 0;
  for (int r = 0; r <= p; ++r) {
    const int c = j + r - op.c0;
    if (c < 0 || c >= op.in.n[axis]) continue;
    acc += v[r] * in[base + (long long)c * sc];
  }
  return acc;
}

template <typename T, typename TOut, int AXIS>
__global__ void k_expand(LayoutDev L, const AxisOp* ops, const T* __restrict__ in, TOut* __restrict__ out,
                         TileMap tm) {
  int opi;
  long long idx0;
  tile_of(tm, opi, idx0);
  const AxisOp& op = block_op(ops, opi);
  const long long nout = (long long)op.out.n[0] * op.out.n[1] * op.out.n[2];
  // with a tile map every thread has one element; else a grid-stride loop
  const long long stride = tm.op ? nout : (long long)gridDim.x * blockDim.x;
  for (long long idx = idx0; idx < nout; idx += stride) {
    int o[3];
    unflatten(idx, op.out.n, o);
    const T val = expand_one<T, AXIS>(L.ax[AXIS], op, o, in);
    const View& ov = op.out;
    out[ov.off + o[0] * ov.st[0] + o[1] * ov.st[1] + o[2] * ov.st[2]] = (TOut)val;
  }
}

// Accumulation of the residual E = q - value of the fused last decode axis.
// FP32 data against float-float values stay on the FP32 pipes (the FP64 pipe
// of this GPU is a small fraction of them): E = (q - hi) - lo, where q - hi is
// exact once the fit is close (Sterbenz); E^2 is the exact FMA product summed
// as a float-float, and the warp reduction moves float-floats.  Any FP64
// operand keeps the FP64 form.
template <typename T, typename TQ>
struct ResidAcc {
  double s2 = 0.0, emax = 0.0, qmin = INFINITY, qmax = -INFINITY;
  __device__ __forceinline__ void add(TQ q, T v) {
    const double qv = (double)q;
    const double e = qv - (double)v;
    s2 += e * e;
    emax = fmax(emax, fabs(e));
    qmin = fmin(qmin, qv);
    qmax = fmax(qmax, qv);
  }
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
      emax = fmax(emax, __shfl_down_sync(0xffffffffu, emax, o));
      qmin = fmin(qmin, __shfl_down_sync(0xffffffffu, qmin, o));
      qmax = fmax(qmax, __shfl_down_sync(0xffffffffu, qmax, o));
    }
  }
  __device__ __forceinline__ double sum2() const { return s2; }
  // block reduction: warp totals through shared memory, merged by one thread
  using Red = double;
  static constexpr int kFields = 4;
  __device__ __forceinline__ void store(Red* sm, int w, int stride) const {
    sm[w] = s2;
    sm[stride + w] = emax;
    sm[2 * stride + w] = qmin;
    sm[3 * stride + w] = qmax;
  }
  __device__ __forceinline__ void merge(const Red* sm, int w, int stride) {
    s2 += sm[w];
    emax = fmax(emax, sm[stride + w]);
    qmin = fmin(qmin, sm[2 * stride + w]);
    qmax = fmax(qmax, sm[3 * stride + w]);
  }
  __device__ __forceinline__ void out(double* o) const {
    o[0] = s2;
    o[1] = emax;
    o[2] = qmin;
    o[3] = qmax;
  }
};

template <>
struct ResidAcc<ff, float> {
  ff s2 = ff(0.f, 0.f);
  float emax = 0.f, qmin = INFINITY, qmax = -INFINITY;
  __device__ __forceinline__ void add(float q, ff v) {
    const float e = __fsub_rn(__fsub_rn(q, v.hi), v.lo);
    const float p = __fmul_rn(e, e);
    s2 += ff(p, __fmaf_rn(e, e, -p));
    emax = fmaxf(emax, fabsf(e));
    qmin = fminf(qmin, q);
    qmax = fmaxf(qmax, q);
  }
  __device__ __forceinline__ void warp_reduce() {
    for (int o = 16; o > 0; o >>= 1) {
      s2 += ff(__shfl_down_sync(0xffffffffu, s2.hi, o), __shfl_down_sync(0xffffffffu, s2.lo, o));
      emax = fmaxf(emax, __shfl_down_sync(0xffffffffu, emax, o));
      qmin = fminf(qmin, __shfl_down_sync(0xffffffffu, qmin, o));
      qmax = fmaxf(qmax, __shfl_down_sync(0xffffffffu, qmax, o));
    }
  }
  __device__ __forceinline__ double sum2() const { return (double)s2.hi + (double)s2.lo; }
  using Red = float;
  static constexpr int kFields = 5;
  __device__ __forceinline__ void store(Red* sm, int w, int stride) const {
    sm[w] = s2.hi;
    sm[stride + w] = s2.lo;
    sm[2 * stride + w] = emax;
    sm[3 * stride + w] = qmin;
    sm[4 * stride + w] = qmax;
  }
  __device__ __forceinline__ void merge(const Red* sm, int w, int stride) {
    s2 += ff(sm[w], sm[stride + w]);
    emax = fmaxf(emax, sm[2 * stride + w]);
    qmin = fminf(qmin, sm[3 * stride + w]);
    qmax = fmaxf(qmax, sm[4 * stride + w]);
  }
  __device__ __forceinline__ void out(double* o) const {
    o[0] = sum2();
    o[1] = emax;
    o[2] = qmin;
    o[3] = qmax;
  }
};

// Batches of independent fits: the last decode axis of a group fused with
// the residual against the data, over a tile map; every tile (one block)
// writes its sum of E^2 and max |E| (ResidAcc, stored as FP64).  Q shares the
// output views.
template <typename T, typename TQ, int AXIS>
__global__ void k_expand_residual_tiles(LayoutDev L, const AxisOp* ops, const T* __restrict__ in,
                                        const TQ* __restrict__ q, TileMap tm, double* __restrict__ tile_part) {
  int opi;
  long long idx;
  tile_of(tm, opi, idx);
  const AxisOp& op = block_op(ops, opi);
  const long long nout = (long long)op.out.n[0] * op.out.n[1] * op.out.n[2];
  ResidAcc<T, TQ> acc;
  if (idx < nout) {
    int o[3];
    unflatten(idx, op.out.n, o);
    const T val = expand_one<T, AXIS>(L.ax[AXIS], op, o, in);
    const View& ov = op.out;
    acc.add(q[ov.off + o[0] * ov.st[0] + o[1] * ov.st[1] + o[2] * ov.st[2]], val);
  }
  acc.warp_reduce();
  using Acc = ResidAcc<T, TQ>;
  __shared__ typename Acc::Red red[Acc::kFields * 32];  // up to 1024 threads
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) acc.store(red, w, 32);
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc tot;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot.merge(red, k, 32);
    double o[4];
    tot.out(o);
    tile_part[2 * blockIdx.x] = o[0];
    tile_part[2 * blockIdx.x + 1] = o[1];
  }
}

// Per-instance totals of the tile partials, tiles in order: instance i of
// the group owns tiles [first[i], first[i+1]); out[2 * id[i]] = sum of E^2,
// out[2 * id[i] + 1] = max |E|.  One warp per instance.
__global__ void k_tiles_to_instances(const double* __restrict__ tile_part, const int* __restrict__ first,
                                     const int* __restrict__ id, int count, double* __restrict__ out) {
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= count) return;
  double a = 0.0, b = 0.0;
  for (int t = first[i] + lane; t < first[i + 1]; t += 32) {
    a += tile_part[2 * t];
    b = fmax(b, tile_part[2 * t + 1]);
  }
  for (int sft = 16; sft > 0; sft >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, sft);
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, sft));
  }
  if (lane == 0) {
    out[2 * id[i]] = a;
    out[2 * id[i] + 1] = b;
  }
}

// the axis is a template argument of the kernels, so every per-axis index of
// an operand view is known at compile time and the view stays in registers
#define MFA_AXIS_DISPATCH(axis, LAUNCH) \
  do {                                  \
    if ((axis) == 0) {                  \
      constexpr int AX = 0;             \
      LAUNCH;                           \
    } else if ((axis) == 1) {           \
      constexpr int AX = 1;             \
      LAUNCH;                           \
    } else {                            \
      constexpr int AX = 2;             \
      LAUNCH;                           \
    }                                   \
  } while (0)

template <typename T, typename TQ>
void launch_expand_residual_tiles(const LayoutDev& L, int axis, const AxisOp* ops, const T* in, const TQ* q,
                                  const TileMap& tm, double* tile_part, const int* first, const int* id, int count,
                                  double* out, cudaStream_t st) {
  if (tm.ntiles > 0)
    MFA_AXIS_DISPATCH(axis, (k_expand_residual_tiles<T, TQ, AX><<<tm.ntiles, tm.threads, 0, st>>>(L, ops, in, q, tm, tile_part)));
  if (count > 0) k_tiles_to_instances<<<(count + 7) / 8, 256, 0, st>>>(tile_part, first, id, count, out);
}

// Final decode axis fused with the residual E = Q - R P: per-block partial
// sums of E^2, max |E|, min Q and max Q (ResidAcc), written as FP64.  Q shares
// the output layout.
template <typename T, typename TQ, int AXIS>
__global__ void k_expand_residual(LayoutDev L, const AxisOp* opp, const T* __restrict__ in,
                                  const TQ* __restrict__ q, double* partials) {
  const AxisOp& op = block_op(opp, 0);
  const long long nout = (long long)op.out.n[0] * op.out.n[1] * op.out.n[2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  ResidAcc<T, TQ> acc;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nout; idx += stride) {
    int o[3];
    unflatten(idx, op.out.n, o);
    acc.add(q[idx], expand_one<T, AXIS>(L.ax[AXIS], op, o, in));
  }
  acc.warp_reduce();
  using Acc = ResidAcc<T, TQ>;
  __shared__ typename Acc::Red sh[Acc::kFields * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) acc.store(sh, wid, 32);
  __syncthreads();
  if (threadIdx.x == 0) {
    Acc tot;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot.merge(sh, i, 32);
    double o[4];
    tot.out(o);
    for (int k = 0; k < 4; ++k) partials[4 * blockIdx.x + k] = o[k];
  }
}

// Fixed-order reduction of per-block partials (deterministic): CTA b reduces
// rows [b * chunk, (b + 1) * chunk) of `partials` into row b of `result`.
__global__ void k_reduce_partials(const double* partials, int nblocks, double* result, int chunk) {
  __shared__ double sh[4][256];
  double a = 0.0, b = 0.0, c = INFINITY, d = -INFINITY;
  const int r0 = blockIdx.x * chunk, r1 = min(nblocks, r0 + chunk);
  result += 4 * blockIdx.x;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    a += partials[4 * i];
    b = fmax(b, partials[4 * i + 1]);
    c = fmin(c, partials[4 * i + 2]);
    d = fmax(d, partials[4 * i + 3]);
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  sh[3][threadIdx.x] = d;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + s]);
      sh[2][threadIdx.x] = fmin(sh[2][threadIdx.x], sh[2][threadIdx.x + s]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) result[i] = sh[i][0];
}

// Banded matrix-vector product along one axis with the output restricted to
// the owned rows: out[i] = sum_c A_L(oU+i, c) in[c], |oU+i-c| <= p.  This is
// the coupling G = N_U^T N_L of the Schur-decoupled local problem.
template <typename T, int AXIS>
__global__ void k_band_apply(LayoutDev L, const AxisOp* ops, const T* __restrict__ in, T* __restrict__ out) {
  constexpr int axis = AXIS;
  const AxisOp& op = block_op(ops, blockIdx.y);
  const long long nout = (long long)op.out.n[0] * op.out.n[1] * op.out.n[2];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nout) return;
  int o[3];
  unflatten(idx, op.out.n, o);
  const AxisDev& ax = L.ax[axis];
  const int p = ax.p, w = p + 1;
  const AxisSub sb = ax.subs[op.sa];
  const double* A = ax.AL + (long long)sb.bandL * w;
  const int r = op.oU + o[axis];
  const int nL = op.in.n[axis];
  long long base = op.in.off;
  for (int a = 0; a < 3; ++a)
    if (a != axis) base += (long long)o[a] * op.in.st[a];
  const long long sc = op.in.st[axis];
  T acc = 0;
  const int c_lo = r - p < 0 ? 0 : r - p;
  const int c_hi = r + p > nL - 1 ? nL - 1 : r + p;
  for (int c = c_lo; c <= c_hi; ++c) {
    const double a = c >= r ? A[(long long)r * w + (c - r)] : A[(long long)c * w + (r - c)];
    acc += (T)a * in[base + (long long)c * sc];
  }
  const View& ov = op.out;
  out[ov.off + o[0] * ov.st[0] + o[1] * ov.st[1] + o[2] * ov.st[2]] = acc;
}

// In-place banded Cholesky solve along one axis, one thread per fibre
// (Sec. 2.3.1): forward L y = c, then backward L^T x = y.  The p values last
// solved stay in registers (a window shifted by one per step), and the next
// right-hand side and factor row are loaded one step ahead, so the recurrence
// waits on arithmetic only; the operations and their order are those of the
// plain substitution.
template <typename T, int AXIS>
__global__ void k_band_solve(LayoutDev L, bool useU, const AxisOp* ops, T* x, TileMap tm) {
  constexpr int axis = AXIS;
  constexpr int PM = MFA_MAX_DEGREE;
  int opi;
  long long f;
  tile_of(tm, opi, f);
  const AxisOp& op = block_op(ops, opi);
  const View& v = op.out;
  const int a1 = axis == 0 ? 1 : 0, a2 = axis == 2 ? 1 : 2;
  const long long nf = (long long)v.n[a1] * v.n[a2];
  if (f >= nf) return;
  const int i1 = (int)(f % v.n[a1]), i2 = (int)(f / v.n[a1]);
  const AxisDev& ax = L.ax[axis];
  const int p = ax.p, w = p + 1;
  const AxisSub sb = ax.subs[op.sa];
  const T* F = useU ? fac_U<T>(ax) + (long long)sb.bandU * w : fac_L<T>(ax) + (long long)sb.bandL * w;
  const int n = v.n[axis];
  T* base = x + v.off + (long long)i1 * v.st[a1] + (long long)i2 * v.st[a2];
  const long long s = v.st[axis];
  T win[PM];  // win[e - 1] = the value solved e steps ago
#pragma unroll
  for (int e = 0; e < PM; ++e) win[e] = T(0.f);
  T Fr[PM + 1];  // factor row of the current step
  T rhs = n > 0 ? base[0] : T(0.f);
#pragma unroll
  for (int e = 0; e <= PM; ++e) Fr[e] = e <= p && n > 0 ? F[e] : T(0.f);
  for (int i = 0; i < n; ++i) {
    // next step's operands, independent of this step's result
    T rhs_n = i + 1 < n ? base[(i + 1) * s] : T(0.f);
    T Fn[PM + 1];
#pragma unroll
    for (int e = 0; e <= PM; ++e) Fn[e] = e <= p && i + 1 < n ? F[(i + 1) * w + e] : T(0.f);
    T acc = rhs;
#pragma unroll
    for (int e = 1; e <= PM; ++e)
      if (e <= p && e <= i) acc -= Fr[e] * win[e - 1];
    const T xi = acc * Fr[0];
    base[i * s] = xi;
#pragma unroll
    for (int e = PM - 1; e > 0; --e) win[e] = win[e - 1];
    win[0] = xi;
    rhs = rhs_n;
#pragma unroll
    for (int e = 0; e <= PM; ++e) Fr[e] = Fn[e];
  }
  // backward: x_i = (y_i - sum_e L(i+e, i) x_{i+e}) / L(i, i); the window
  // holds x_{i+1} .. x_{i+p}, starting from the last forward values
  // (win[0] = y_{n-1}, which is the first value solved backwards)
#pragma unroll
  for (int e = 0; e < PM; ++e) win[e] = T(0.f);
  rhs = n > 0 ? base[(n - 1) * s] : T(0.f);
  for (int i = n - 1; i >= 0; --i) {
    T rhs_n = i > 0 ? base[(i - 1) * s] : T(0.f);
    T acc = rhs;
#pragma unroll
    for (int e = 1; e <= PM; ++e)
      if (e <= p && i + e < n) acc -= F[(i + e) * w + e] * win[e - 1];
    const T xi = acc * F[i * w];
    base[i * s] = xi;
#pragma unroll
    for (int e = PM - 1; e > 0; --e) win[e] = win[e - 1];
    win[0] = xi;
    rhs = rhs_n;
  }
}

template <typename T, typename TIn>
void launch_contract(const LayoutDev& L, int axis, const AxisOp* ops, int nops, int max_out, const TIn* in, T* out,
                     int* status, cudaStream_t st, const TileMap* tm) {
  if (tm && tm->op) {
    if (tm->ntiles > 0) MFA_AXIS_DISPATCH(axis, (k_contract<T, TIn, AX><<<tm->ntiles, tm->threads, 0, st>>>(L, ops, in, out, status, *tm)));
    return;
  }
  dim3 grid((max_out + kContractThreads - 1) / kContractThreads, nops);
  MFA_AXIS_DISPATCH(axis, (k_contract<T, TIn, AX><<<grid, kContractThreads, 0, st>>>(L, ops, in, out, status, TileMap{})));
}

template <typename T, typename TOut>
void launch_expand(const LayoutDev& L, int axis, const AxisOp* ops, int nops, long long max_out, const T* in,
                   TOut* out, cudaStream_t st, const TileMap* tm) {
  if (tm && tm->op) {
    if (tm->ntiles > 0) MFA_AXIS_DISPATCH(axis, (k_expand<T, TOut, AX><<<tm->ntiles, tm->threads, 0, st>>>(L, ops, in, out, *tm)));
    return;
  }
  long long blocks = (max_out + kExpandThreads - 1) / kExpandThreads;
  if (blocks > 65535) blocks = 65535;
  dim3 grid((unsigned)blocks, nops);
  MFA_AXIS_DISPATCH(axis, (k_expand<T, TOut, AX><<<grid, kExpandThreads, 0, st>>>(L, ops, in, out, TileMap{})));
}

template <typename T, typename TQ>
void launch_expand_residual(const LayoutDev& L, int axis, const AxisOp* op, long long /*nout*/, const T* in,
                            const TQ* q, double* partials, int nblocks, cudaStream_t st) {
  MFA_AXIS_DISPATCH(axis, (k_expand_residual<T, TQ, AX><<<nblocks, 256, 0, st>>>(L, op, in, q, partials)));
}

void launch_reduce_partials(const double* partials, int nblocks, double* result, cudaStream_t st, double* scratch,
                            int scratch_rows) {
  // two fixed-order passes when there are many partials: chunks on many SMs,
  // then one CTA over the chunk results
  const int R = std::min(128, scratch_rows);
  if (scratch && nblocks > 8 * 256 && R > 1) {
    const int chunk = (nblocks + R - 1) / R;
    k_reduce_partials<<<R, 256, 0, st>>>(partials, nblocks, scratch, chunk);
    k_reduce_partials<<<1, 256, 0, st>>>(scratch, R, result, R);
  } else {
    k_reduce_partials<<<1, 256, 0, st>>>(partials, nblocks, result, nblocks);
  }
}

template <typename T>
void launch_band_apply(const LayoutDev& L, int axis, const AxisOp* ops, int nops, int max_out, const T* in, T* out,
                       cudaStream_t st) {
  dim3 grid((max_out + 127) / 128, nops);
  MFA_AXIS_DISPATCH(axis, (k_band_apply<T, AX><<<grid, 128, 0, st>>>(L, ops, in, out)));
}

template <typename T>
void launch_band_solve(const LayoutDev& L, int axis, bool useU, const AxisOp* ops, int nops, int max_fibres, T* x,
                       cudaStream_t st, const TileMap* tm) {
  if (tm && tm->op) {
    if (tm->ntiles > 0) MFA_AXIS_DISPATCH(axis, (k_band_solve<T, AX><<<tm->ntiles, tm->threads, 0, st>>>(L, useU, ops, x, *tm)));
    return;
  }
  dim3 grid((max_fibres + kSolveThreads - 1) / kSolveThreads, nops);
  MFA_AXIS_DISPATCH(axis, (k_band_solve<T, AX><<<grid, kSolveThreads, 0, st>>>(L, useU, ops, x, TileMap{})));
}

#define MFA_INST_T(T)                                                                                        \
  template void launch_band_apply<T>(const LayoutDev&, int, const AxisOp*, int, int, const T*, T*, cudaStream_t);   \
  template void launch_band_solve<T>(const LayoutDev&, int, bool, const AxisOp*, int, int, T*, cudaStream_t,       \
                                     const TileMap*);                                                            \
  template void launch_contract<T, float>(const LayoutDev&, int, const AxisOp*, int, int, const float*, T*, int*,  \
                                          cudaStream_t, const TileMap*);                                           \
  template void launch_contract<T, double>(const LayoutDev&, int, const AxisOp*, int, int, const double*, T*, int*, \
                                           cudaStream_t, const TileMap*);                                          \
  template void launch_expand_residual<T, float>(const LayoutDev&, int, const AxisOp*, long long, const T*,        \
                                                 const float*, double*, int, cudaStream_t);                        \
  template void launch_expand_residual<T, double>(const LayoutDev&, int, const AxisOp*, long long, const T*,       \
                                                  const double*, double*, int, cudaStream_t);                      \
  template void launch_expand<T, float>(const LayoutDev&, int, const AxisOp*, int, long long, const T*, float*,    \
                                        cudaStream_t, const TileMap*);                                             \
  template void launch_expand<T, double>(const LayoutDev&, int, const AxisOp*, int, long long, const T*, double*,  \
                                         cudaStream_t, const TileMap*);

MFA_INST_T(double)
MFA_INST_T(float)
MFA_INST_T(ff)
template void launch_expand_residual_tiles<double, float>(const LayoutDev&, int, const AxisOp*, const double*,
                                                          const float*, const TileMap&, double*, const int*,
                                                          const int*, int, double*, cudaStream_t);
template void launch_expand_residual_tiles<double, double>(const LayoutDev&, int, const AxisOp*, const double*,
                                                           const double*, const TileMap&, double*, const int*,
                                                           const int*, int, double*, cudaStream_t);
template void launch_expand_residual_tiles<ff, float>(const LayoutDev&, int, const AxisOp*, const ff*, const float*,
                                                      const TileMap&, double*, const int*, const int*, int, double*,
                                                      cudaStream_t);
template void launch_expand_residual_tiles<ff, double>(const LayoutDev&, int, const AxisOp*, const ff*,
                                                       const double*, const TileMap&, double*, const int*,
                                                       const int*, int, double*, cudaStream_t);
template void launch_expand<ff, ff>(const LayoutDev&, int, const AxisOp*, int, long long, const ff*, ff*,
                                    cudaStream_t, const TileMap*);
template void launch_contract<ff, ff>(const LayoutDev&, int, const AxisOp*, int, int, const ff*, ff*, int*,
                                      cudaStream_t, const TileMap*);

}  // namespace mfa
