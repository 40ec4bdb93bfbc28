// Schwarz exchange and update kernels (Sec. 2.3.2, Algorithm 1 loop body) and
// scattered decode.
#include "mfa_internal.cuh"

#include <type_traits>

namespace mfa {

struct SubBox {
  int l0[3], nL[3], oU[3], nU[3];
};

__device__ __forceinline__ SubBox sub_box(const LayoutDev& L, int s) {
  SubBox b;
  int r = s;
  for (int a = 0; a < 3; ++a) {
    const int sa = r % L.S[a];
    r /= L.S[a];
    const AxisSub sb = L.ax[a].subs[sa];
    b.l0[a] = sb.l0;
    b.nL[a] = sb.nL;
    b.oU[a] = sb.oU;
    b.nU[a] = sb.nU;
  }
  return b;
}

// Exchange (Algorithm 1: dequeue incoming constraints): every subdomain reads
// the lagged global iterate on its frame F = L \ U; owned entries are zeroed
// so that the coupling product below only sees the fixed frame values.
template <typename T>
__global__ void k_frame_gather(LayoutDev L, const long long* offL, const T* __restrict__ P, T* __restrict__ Pt) {
  const int s = blockIdx.y;
  const SubBox b = sub_box(L, s);
  const long long n = (long long)b.nL[0] * b.nL[1] * b.nL[2];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int i0 = (int)(idx % b.nL[0]);
  const long long r = idx / b.nL[0];
  const int i1 = (int)(r % b.nL[1]), i2 = (int)(r / b.nL[1]);
  const bool owned = i0 >= b.oU[0] && i0 < b.oU[0] + b.nU[0] && i1 >= b.oU[1] && i1 < b.oU[1] + b.nU[1] &&
                     i2 >= b.oU[2] && i2 < b.oU[2] + b.nU[2];
  T v = 0;
  if (!owned) {
    const long long g = (long long)(b.l0[0] + i0) + L.ncp[0] * ((long long)(b.l0[1] + i1) + L.ncp[1] * (b.l0[2] + i2));
    v = P[g];
  }
  Pt[offL[s] + idx] = v;
}

// Right-hand side of the constrained local problem (Schur decoupling):
// X[U] = B_U - (G_0 x G_1 x G_2) P_F, written into the owned box of X.
template <typename T>
__global__ void k_rhs_finalize(LayoutDev L, const long long* offL, const long long* offY, const T* __restrict__ BL,
                               const T* __restrict__ Y, T* __restrict__ X) {
  const int s = blockIdx.y;
  const SubBox b = sub_box(L, s);
  const long long n = (long long)b.nU[0] * b.nU[1] * b.nU[2];
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int i0 = (int)(idx % b.nU[0]);
  const long long r = idx / b.nU[0];
  const int i1 = (int)(r % b.nU[1]), i2 = (int)(r / b.nU[1]);
  const long long li =
      (long long)(i0 + b.oU[0]) + (long long)b.nL[0] * ((long long)(i1 + b.oU[1]) + (long long)b.nL[1] * (i2 + b.oU[2]));
  X[offL[s] + li] = BL[offL[s] + li] - Y[offY[s] + idx];
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Update (Sec. 2.3.2): P^k(g) = (1/n_s) sum over the owned copies of g, read in
// a fixed order (deterministic).  Also accumulates max|P^k - P^{k-1}|, max|P^k|
// and the largest copy spread (jump residual) into metrics[0..2] as the bit
// patterns of non-negative doubles.
template <typename T>
__global__ void k_average(LayoutDev L, const long long* offL, const T* __restrict__ X, T* __restrict__ P,
                          const T* __restrict__ Pprev, unsigned long long* metrics, int rule) {
  const long long n = L.ncp[0] * L.ncp[1] * L.ncp[2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  double dmax = 0.0, pmax = 0.0, spread = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += stride) {
    int gi[3];
    gi[0] = (int)(g % L.ncp[0]);
    const long long r = g / L.ncp[0];
    gi[1] = (int)(r % L.ncp[1]);
    gi[2] = (int)(r / L.ncp[1]);
    int f[3], c[3];
    for (int a = 0; a < 3; ++a) {
      f[a] = L.ax[a].own_first[gi[a]];
      c[a] = L.ax[a].own_count[gi[a]];
    }
    double sum = 0.0, lo = INFINITY, hi = -INFINITY;
    int cnt = 0;
    T owner_val = T(0);
    for (int c2 = 0; c2 < c[2]; ++c2)
      for (int c1 = 0; c1 < c[1]; ++c1)
        for (int c0 = 0; c0 < c[0]; ++c0) {
          const int sa0 = f[0] + c0, sa1 = f[1] + c1, sa2 = f[2] + c2;
          const int s = sa0 + L.S[0] * (sa1 + L.S[1] * sa2);
          const AxisSub b0 = L.ax[0].subs[sa0], b1 = L.ax[1].subs[sa1], b2 = L.ax[2].subs[sa2];
          const long long li = (long long)(gi[0] - b0.l0) +
                               (long long)b0.nL * ((long long)(gi[1] - b1.l0) + (long long)b1.nL * (gi[2] - b2.l0));
          const T xv = X[offL[s] + li];
          const double v = (double)xv;
          if (c0 == L.ax[0].own_pick[gi[0]] && c1 == L.ax[1].own_pick[gi[1]] && c2 == L.ax[2].own_pick[gi[2]])
            owner_val = xv;
          sum += v;
          lo = fmin(lo, v);
          hi = fmax(hi, v);
          ++cnt;
        }
    const T pn = rule == UPDATE_OWNER ? owner_val : (T)(sum / cnt);
    P[g] = pn;
    pmax = fmax(pmax, fabs((double)pn));
    spread = fmax(spread, hi - lo);
    if (Pprev) dmax = fmax(dmax, fabs((double)pn - (double)Pprev[g]));
  }
  for (int off = 16; off > 0; off >>= 1) {
    dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
    pmax = fmax(pmax, __shfl_down_sync(0xffffffffu, pmax, off));
    spread = fmax(spread, __shfl_down_sync(0xffffffffu, spread, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&metrics[0], dmax);
    atomic_max_nonneg(&metrics[1], pmax);
    atomic_max_nonneg(&metrics[2], spread);
  }
}

template <typename T>
void launch_frame_gather(const LayoutDev& L, const long long* offL, int maxL, const T* P, T* Pt, cudaStream_t st) {
  dim3 grid((maxL + 127) / 128, L.nsub);
  k_frame_gather<T><<<grid, 128, 0, st>>>(L, offL, P, Pt);
}

template <typename T>
void launch_rhs_finalize(const LayoutDev& L, const long long* offL, const long long* offY, int maxU, const T* BL,
                         const T* Y, T* X, cudaStream_t st) {
  dim3 grid((maxU + 127) / 128, L.nsub);
  k_rhs_finalize<T><<<grid, 128, 0, st>>>(L, offL, offY, BL, Y, X);
}

template <typename T>
void launch_average(const LayoutDev& L, const long long* offL, const T* X, T* P, const T* Pprev,
                    unsigned long long* metrics, cudaStream_t st, int rule) {
  const long long n = L.ncp[0] * L.ncp[1] * L.ncp[2];
  long long blocks = (n + 255) / 256;
  const long long cap = 16LL * device_sm_count();
  if (blocks > cap) blocks = cap;
  k_average<T><<<(unsigned)blocks, 256, 0, st>>>(L, offL, X, P, Pprev, metrics, rule);
}

// ---------------------------------------------------------------------------
// Scattered decode with derivatives (Sec. 2.1: exact derivatives from the
// Cox-de Boor recurrence).
// ---------------------------------------------------------------------------

__device__ __forceinline__ double knot_at2(int i, int p, int nspans) {
  if (i <= p) return 0.0;
  if (i >= nspans + p) return 1.0;
  return (double)(i - p) / (double)nspans;
}

// Values of the order-`r` derivatives of the p+1 degree-p functions nonzero on
// span j at u.  First the degree p-r functions by the value recurrence, then r
// steps of the derivative recurrence
//   d/du N_{m,q} = q/(t_{m+q}-t_m) N_{m,q-1} - q/(t_{m+q+1}-t_{m+1}) N_{m+1,q-1}
// (with the lower-degree functions already differentiated r-1 times).
__device__ void basis_derivs(int j, double u, int p, int nspans, int rder, double* N) {
  const int i = j + p;
  const int q0 = p - rder;
  for (int r = 0; r <= p; ++r) N[r] = 0.0;
  if (q0 < 0) return;
  N[0] = 1.0;
  for (int q = 1; q <= q0; ++q) {
    double carry = 0.0;
    for (int r = 0; r < q; ++r) {
      const double tl = knot_at2(i - q + r + 1, p, nspans);
      const double tr = knot_at2(i + r + 1, p, nspans);
      const double w = N[r] / (tr - tl);
      const double right = (tr - u) * w;
      const double left_next = (u - tl) * w;
      N[r] = carry + right;
      carry = left_next;
    }
    N[q] = carry;
  }
  for (int q = q0 + 1; q <= p; ++q) {
    double carry = 0.0;
    for (int r = 0; r < q; ++r) {
      const double tl = knot_at2(i - q + r + 1, p, nspans);
      const double tr = knot_at2(i + r + 1, p, nspans);
      const double w = q * N[r] / (tr - tl);
      N[r] = carry - w;  // -q/(t_{m+q+1}-t_{m+1}) N_{m+1,q-1} for m = i-q+r
      carry = w;         // +q/(t_{m+q}-t_m) N_{m,q-1} for m = i-q+r+1
    }
    N[q] = carry;
  }
}

// Derivatives of order rder (with respect to u) of the p+1 basis functions of
// axis `ax` nonzero at u, into N; returns the first one's control point.
// Floating knots: the global clamped uniform knots.  Clamped interfaces: the
// core holding u and its own clamped uniform knots of b - a spans at the local
// parameter (x - a)/(b - a), x = u * gspans, so each derivative order takes a
// factor gspans / (b - a).  With weights, the rational basis R = N W / w
// (Eq. nurbs-basis) and its derivatives from differentiating w R = N W r times
// (Leibniz): R^(r) = (N^(r) W - sum_{j=1..r} binom(r, j) w^(j) R^(r-j)) / w,
// w^(j) = sum N^(j) W.
__device__ int axis_basis(const AxisDev& ax, double u, int rder, double* N) {
  const int p = ax.p;
  int first, ns, j;
  double ul, dscale = 1.0;
  if (ax.kmode == KMODE_CLAMPED) {
    const int gs = ax.gspans;
    const double x = u * gs;
    int jg = (int)floor(x);
    jg = jg > gs - 1 ? gs - 1 : (jg < 0 ? 0 : jg);
    int lo = 0, hi = ax.S - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ax.subs[mid].a <= jg) lo = mid;
      else hi = mid - 1;
    }
    const AxisSub sb = ax.subs[lo];
    ns = sb.b - sb.a;
    j = jg - sb.a;
    ul = (x - (double)sb.a) / (double)ns;
    first = sb.l0 + sb.oU + j;
    dscale = (double)gs / (double)ns;
  } else {
    ns = ax.nspans;
    j = (int)floor(u * ns);
    j = j > ns - 1 ? ns - 1 : (j < 0 ? 0 : j);
    ul = u;
    first = j;
  }
  if (!ax.wts) {
    basis_derivs(j, ul, p, ns, rder, N);
    double f = 1.0;
    for (int r = 0; r < rder; ++r) f *= dscale;
    for (int r = 0; r <= p; ++r) N[r] *= f;
    return first;
  }
  double R[MFA_MAX_DEGREE + 1][MFA_MAX_DEGREE + 1], w[MFA_MAX_DEGREE + 1];
  double f = 1.0;
  for (int i = 0; i <= rder; ++i) {
    basis_derivs(j, ul, p, ns, i, R[i]);
    w[i] = 0.0;
    for (int r = 0; r <= p; ++r) {
      R[i][r] *= f * ax.wts[first + r];  // N^(i) W
      w[i] += R[i][r];
    }
    f *= dscale;
  }
  for (int i = 0; i <= rder; ++i) {
    double binom = 1.0;  // binom(i, jj)
    for (int jj = 1; jj <= i; ++jj) {
      binom = binom * (i - jj + 1) / jj;
      for (int r = 0; r <= p; ++r) R[i][r] -= binom * w[jj] * R[i - jj][r];
    }
    for (int r = 0; r <= p; ++r) R[i][r] /= w[0];
  }
  for (int r = 0; r <= p; ++r) N[r] = R[rder][r];
  return first;
}

template <typename T>
__global__ void k_decode_points(LayoutDev L, double lo0, double lo1, double lo2, double hi0, double hi1, double hi2,
                                const double* __restrict__ pts, long long npts, int d0, int d1, int d2,
                                const T* __restrict__ P, void* out, int out_dtype) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
  const int der[3] = {d0, d1, d2};
  double N[3][MFA_MAX_DEGREE + 1];
  int span[3];
  double scale = 1.0;
  for (int a = 0; a < 3; ++a) {
    const AxisDev& ax = L.ax[a];
    double u = 0.0;
    if (a < L.dim) {
      const double len = hi[a] - lo[a];
      u = len != 0.0 ? (pts[k * L.dim + a] - lo[a]) / len : 0.0;
      u = fmin(fmax(u, 0.0), 1.0);
      for (int r = 0; r < der[a]; ++r) scale /= len;
    }
    span[a] = axis_basis(ax, u, a < L.dim ? der[a] : 0, N[a]);
  }
  double acc = 0.0;
  for (int r2 = 0; r2 <= L.ax[2].p; ++r2) {
    double acc1 = 0.0;
    for (int r1 = 0; r1 <= L.ax[1].p; ++r1) {
      double acc0 = 0.0;
      const long long row = (long long)(span[1] + r1) * L.ncp[0] + (long long)(span[2] + r2) * L.ncp[0] * L.ncp[1];
      for (int r0 = 0; r0 <= L.ax[0].p; ++r0) acc0 += N[0][r0] * (double)P[row + span[0] + r0];
      acc1 += N[1][r1] * acc0;
    }
    acc += N[2][r2] * acc1;
  }
  acc *= scale;
  if (out_dtype == MFA_F64)
    ((double*)out)[k] = acc;
  else
    ((float*)out)[k] = (float)acc;
}

void launch_decode_points_ff(const LayoutDev& L, const double* lo, const double* hi, const double* pts,
                             long long npts, const int* deriv, const ff* P, void* out, int out_dtype, cudaStream_t st);

template <typename T>
void launch_decode_points(const LayoutDev& L, const double* lo, const double* hi, const double* pts, long long npts,
                          const int* deriv, const T* P, void* out, int out_dtype, cudaStream_t st) {
  if constexpr (std::is_same<T, ff>::value) {
    launch_decode_points_ff(L, lo, hi, pts, npts, deriv, P, out, out_dtype, st);
  } else {
    long long blocks = (npts + 127) / 128;
    k_decode_points<T><<<(unsigned)blocks, 128, 0, st>>>(L, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], pts, npts,
                                                         deriv[0], deriv[1], deriv[2], P, out, out_dtype);
  }
}

// Scattered decode of instances of a batch of independent fits: point k
// belongs to query q with pt_off[q] <= k < pt_off[q+1], which evaluates
// instance qinst[q]; coordinates are parameters u in [0,1] per axis (stride
// 3, clamped), the value is sum over the (p+1)^dim control points of the
// tensor-product basis (Sec. 2.1) in FP64.
template <typename T>
__global__ void k_decode_points_inst(const InstDesc* __restrict__ desc, const int* __restrict__ qinst,
                                     const long long* __restrict__ pt_off, int nq, const double* __restrict__ pts,
                                     const T* __restrict__ P, double* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= pt_off[nq]) return;
  int lo = 0, hi = nq - 1;  // last query whose first point is <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pt_off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  const InstDesc D = desc[qinst[lo]];
  double N[3][MFA_MAX_DEGREE + 1];
  int span[3], pa[3];
  for (int a = 0; a < 3; ++a) {
    if (a < D.dim) {
      const double u = fmin(fmax(pts[3 * k + a], 0.0), 1.0);
      int j = (int)floor(u * D.nspans[a]);
      if (j > D.nspans[a] - 1) j = D.nspans[a] - 1;
      if (j < 0) j = 0;
      span[a] = j;
      pa[a] = D.p;
      basis_derivs(j, u, D.p, D.nspans[a], 0, N[a]);
    } else {
      span[a] = 0;
      pa[a] = 0;
      N[a][0] = 1.0;
    }
  }
  const long long n0 = D.n[0], n01 = (long long)D.n[0] * D.n[1];
  double acc = 0.0;
  for (int r2 = 0; r2 <= pa[2]; ++r2) {
    double acc1 = 0.0;
    for (int r1 = 0; r1 <= pa[1]; ++r1) {
      double acc0 = 0.0;
      const long long row = D.cp_off + (long long)(span[1] + r1) * n0 + (long long)(span[2] + r2) * n01;
      for (int r0 = 0; r0 <= pa[0]; ++r0) acc0 += N[0][r0] * (double)P[row + span[0] + r0];
      acc1 += N[1][r1] * acc0;
    }
    acc += N[2][r2] * acc1;
  }
  out[k] = acc;
}

void launch_decode_points_inst_ff(const InstDesc* desc, const int* qinst, const long long* pt_off, int nq,
                                  long long npts, const double* pts, const ff* P, double* out, int p_uniform,
                                  cudaStream_t st);

template <typename T>
void launch_decode_points_inst(const InstDesc* desc, const int* qinst, const long long* pt_off, int nq,
                               long long npts, const double* pts, const T* P, double* out, int p_uniform,
                               cudaStream_t st) {
  if (npts <= 0 || nq <= 0) return;
  if constexpr (std::is_same<T, ff>::value)
    launch_decode_points_inst_ff(desc, qinst, pt_off, nq, npts, pts, P, out, p_uniform, st);
  else
    k_decode_points_inst<T><<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out);
}

template void launch_decode_points_inst<double>(const InstDesc*, const int*, const long long*, int, long long,
                                                const double*, const double*, double*, int, cudaStream_t);
template void launch_decode_points_inst<ff>(const InstDesc*, const int*, const long long*, int, long long,
                                            const double*, const ff*, double*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Scattered decode of float-float control points on the FP32 pipes.
//
// The recurrences are those of basis_derivs, taken in knot units: with x =
// u * nspans, the clamped uniform knots are the integers K(i) = clamp(i - p,
// 0, nspans) and a point of span j sits at x = j + t, 0 <= t <= 1.  Every
// denominator of the recurrence is then a difference of two knots bounding
// span j, an integer 1..q, so each division is a product with a float-float
// reciprocal, and the FP64 pipe (1/64 of the FP32 rate here) is used only to
// split the FP64 coordinate and to widen the result.  Derivatives come out
// with respect to x; the caller scales by nspans^r per axis.
// ---------------------------------------------------------------------------

// 1/d for a small positive integer d as a float-float: the rounded float
// reciprocal r and (1 - r d) / d, whose numerator the FMA forms exactly
__device__ __forceinline__ ff ff_rcp_int(int d) {
  const float df = (float)d;
  const float r = __frcp_rn(df);
  const float e = __fmaf_rn(-r, df, 1.f);
  return ff(r, __fmul_rn(e, r));
}

// k - t and t - k for a small integer k
__device__ __forceinline__ ff ff_int_minus(int k, ff t) {
  const ff s = two_sum((float)k, -t.hi);
  return fast_two_sum(s.hi, __fsub_rn(s.lo, t.lo));
}
__device__ __forceinline__ ff ff_minus_int(ff t, int k) {
  const ff s = two_sum(t.hi, -(float)k);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

// Knot span j of the knot coordinate xk (clamped to [0, nspans], NaN to 0)
// and its offset t = xk - j as a float-float.  The split into float words
// rounds xk to about 48 bits.
__device__ __forceinline__ int knot_span_ff(double xk, int nspans, ff& t) {
  float h = __double2float_rn(xk);
  float l = __double2float_rn(xk - (double)h);
  const float ns = (float)nspans;
  if (!(h > 0.f) && !(h == 0.f && l >= 0.f)) h = l = 0.f;  // negative or NaN
  if (h > ns || (h == ns && l > 0.f)) {
    h = ns;
    l = 0.f;
  }
  const float jf = floorf(h);
  int j = (int)jf;
  if (h == jf && l < 0.f) --j;
  j = min(max(j, 0), nspans - 1);
  // h - j is exact: j <= h <= j + 1 and either j = 0 or h <= 2j; |l| is
  // below half an ulp of h and h - j is 0 or a multiple of that ulp
  t = fast_two_sum(__fsub_rn(h, (float)j), l);
  return j;
}

// Degree of a decode instantiation: P > 0 fixes it at compile time (every
// loop unrolled, the basis in registers); P = 0 takes the runtime degree p
// (loops kept, arrays sized for MFA_MAX_DEGREE).
template <int P>
struct DegreeOf {
  static constexpr int kLen = P > 0 ? P + 1 : MFA_MAX_DEGREE + 1;
  static constexpr int kUnroll = P > 0 ? P + 1 : 1;
};

// Values (rder = 0) or order-rder derivatives in x of the p+1 degree-p
// functions nonzero on span j at x = j + t (Sec. 2.1, Cox-de Boor).
template <int P>
__device__ __forceinline__ void basis_derivs_ff(int j, ff t, int p_rt, int nspans, int rder,
                                                ff (&N)[DegreeOf<P>::kLen]) {
  constexpr int U = DegreeOf<P>::kUnroll;
  const int p = P > 0 ? P : p_rt;
  const int q0 = p - rder;
#pragma unroll U
  for (int r = 0; r <= p; ++r) N[r] = ff(0.f, 0.f);
  if (q0 < 0) return;
  N[0] = ff(1.f, 0.f);
#pragma unroll U
  for (int q = 1; q <= p; ++q) {
    ff carry(0.f, 0.f);
#pragma unroll U
    for (int r = 0; r < q; ++r) {
      const int kl = max(r + 1 - q, -j);     // knot K(j + p + r + 1 - q) - j
      const int kr = min(r + 1, nspans - j);  // knot K(j + p + r + 1) - j
      const ff w = N[r] * ff_rcp_int(kr - kl);
      if (q <= q0) {
        N[r] = carry + ff_int_minus(kr, t) * w;
        carry = ff_minus_int(t, kl) * w;
      } else {
        const ff wq = w * ff((float)q, 0.f);
        N[r] = carry - wq;
        carry = wq;
      }
    }
    N[q] = carry;
  }
}

// Sum of the (p+1)^DIM basis products with the control points of the
// support, x fastest; `row0` points at control point (span0, span1, span2).
template <int P, int DIM>
__device__ __forceinline__ ff tensor_sum_ff(const ff* __restrict__ row0, long long n0, long long n01, int p_rt,
                                            const ff (&N)[3][DegreeOf<P>::kLen]) {
  constexpr int U = DegreeOf<P>::kUnroll;
  const int p = P > 0 ? P : p_rt;
  const int R1 = DIM > 1 ? p : 0, R2 = DIM > 2 ? p : 0;
  ff acc(0.f, 0.f);
#pragma unroll U
  for (int r2 = 0; r2 <= R2; ++r2) {
    ff acc1(0.f, 0.f);
#pragma unroll U
    for (int r1 = 0; r1 <= R1; ++r1) {
      const ff* row = row0 + r1 * n0 + r2 * n01;
      ff acc0(0.f, 0.f);
#pragma unroll U
      for (int r0 = 0; r0 <= p; ++r0) ff_acc_prod(acc0, N[0][r0].hi, N[0][r0].lo, row[r0]);
      acc0 = ff_norm(acc0);
      if (DIM > 1)
        ff_acc_prod(acc1, N[1][r1].hi, N[1][r1].lo, acc0);
      else
        acc1 = acc0;
    }
    acc1 = ff_norm(acc1);
    if (DIM > 2)
      ff_acc_prod(acc, N[2][r2].hi, N[2][r2].lo, acc1);
    else
      acc = acc1;
  }
  return ff_norm(acc);
}

// One point: knot coordinates xk[a] (a < dim), derivative orders der[a].
template <int P>
__device__ __forceinline__ ff decode_point_ff(int dim, int p_rt, const double (&xk)[3], const int (&ns)[3],
                                              const int (&der)[3], const ff* __restrict__ Pc, long long n0,
                                              long long n01) {
  ff N[3][DegreeOf<P>::kLen];
  int span[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      ff t;
      span[a] = knot_span_ff(xk[a], ns[a], t);
      basis_derivs_ff<P>(span[a], t, p_rt, ns[a], der[a], N[a]);
    }
  }
  const ff* row0 = Pc + span[0] + span[1] * n0 + span[2] * n01;
  if (dim == 3) return tensor_sum_ff<P, 3>(row0, n0, n01, p_rt, N);
  if (dim == 2) return tensor_sum_ff<P, 2>(row0, n0, n01, p_rt, N);
  return tensor_sum_ff<P, 1>(row0, n0, n01, p_rt, N);
}

// Batch instances (same indexing as k_decode_points_inst), one point per
// thread; P > 0 when every instance of the batch has degree P.
template <int P>
__global__ void k_decode_points_inst_ff(const InstDesc* __restrict__ desc, const int* __restrict__ qinst,
                                        const long long* __restrict__ pt_off, int nq, const double* __restrict__ pts,
                                        const ff* __restrict__ Pc, double* __restrict__ out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= pt_off[nq]) return;
  int lo = 0, hi = nq - 1;  // last query whose first point is <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pt_off[mid] <= k) lo = mid;
    else hi = mid - 1;
  }
  const InstDesc D = desc[qinst[lo]];
  const double* u = pts + 3 * k;
  const double xk[3] = {u[0] * D.nspans[0], u[1] * D.nspans[1], u[2] * D.nspans[2]};
  const int der[3] = {0, 0, 0};
  const ff v = decode_point_ff<P>(D.dim, D.p, xk, D.nspans, der, Pc + D.cp_off, D.n[0], (long long)D.n[0] * D.n[1]);
  out[k] = (double)v.hi + (double)v.lo;
}

void launch_decode_points_inst_ff(const InstDesc* desc, const int* qinst, const long long* pt_off, int nq,
                                  long long npts, const double* pts, const ff* P, double* out, int p_uniform,
                                  cudaStream_t st) {
  const unsigned blocks = (unsigned)((npts + 127) / 128);
  switch (p_uniform) {
    case 1: k_decode_points_inst_ff<1><<<blocks, 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out); break;
    case 2: k_decode_points_inst_ff<2><<<blocks, 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out); break;
    case 3: k_decode_points_inst_ff<3><<<blocks, 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out); break;
    case 4: k_decode_points_inst_ff<4><<<blocks, 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out); break;
    default: k_decode_points_inst_ff<0><<<blocks, 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out); break;
  }
}

// Model points in the model's coordinates: x_k = (pts - lo) * s with s =
// nspans / (hi - lo) per axis; the derivative scale is formed on the host.
struct PointMap {
  double lo[3], s[3];
  int ns[3], der[3];
  long long n0, n01;
  int dim, p;
  double scale;
};

template <int P>
__global__ void k_decode_points_ff(PointMap m, const double* __restrict__ pts, long long npts,
                                   const ff* __restrict__ Pc, void* __restrict__ out, int out_dtype) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npts) return;
  double xk[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < m.dim) xk[a] = (pts[k * m.dim + a] - m.lo[a]) * m.s[a];
  const ff v = decode_point_ff<P>(m.dim, m.p, xk, m.ns, m.der, Pc, m.n0, m.n01);
  if (m.scale != 1.0) {
    const double d = ((double)v.hi + (double)v.lo) * m.scale;
    if (out_dtype == MFA_F64)
      ((double*)out)[k] = d;
    else
      ((float*)out)[k] = (float)d;
  } else if (out_dtype == MFA_F64) {
    ((double*)out)[k] = (double)v.hi + (double)v.lo;
  } else {
    ((float*)out)[k] = __fadd_rn(v.hi, v.lo);
  }
}

void launch_decode_points_ff(const LayoutDev& L, const double* lo, const double* hi, const double* pts,
                             long long npts, const int* deriv, const ff* P, void* out, int out_dtype, cudaStream_t st) {
  if (npts <= 0) return;
  PointMap m;
  m.dim = L.dim;
  m.p = L.ax[0].p;
  m.scale = 1.0;
  for (int a = 0; a < 3; ++a) {
    const bool on = a < L.dim;
    const double len = on ? hi[a] - lo[a] : 0.0;
    m.lo[a] = on ? lo[a] : 0.0;
    m.ns[a] = L.ax[a].nspans;
    m.s[a] = len != 0.0 ? (double)m.ns[a] / len : 0.0;
    m.der[a] = on ? deriv[a] : 0;
    for (int r = 0; r < m.der[a]; ++r) m.scale *= (double)m.ns[a] / len;  // d/du = nspans d/dx, u = (x - lo) / len
  }
  m.n0 = L.ncp[0];
  m.n01 = (long long)L.ncp[0] * L.ncp[1];
  const unsigned blocks = (unsigned)((npts + 127) / 128);
  switch (m.p) {
    case 1: k_decode_points_ff<1><<<blocks, 128, 0, st>>>(m, pts, npts, P, out, out_dtype); break;
    case 2: k_decode_points_ff<2><<<blocks, 128, 0, st>>>(m, pts, npts, P, out, out_dtype); break;
    case 3: k_decode_points_ff<3><<<blocks, 128, 0, st>>>(m, pts, npts, P, out, out_dtype); break;
    case 4: k_decode_points_ff<4><<<blocks, 128, 0, st>>>(m, pts, npts, P, out, out_dtype); break;
    default: k_decode_points_ff<0><<<blocks, 128, 0, st>>>(m, pts, npts, P, out, out_dtype); break;
  }
}

template <typename TIn, typename TOut>
__global__ void k_cast(const TIn* in, TOut* out, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (TOut)in[i];
}

template <typename TIn, typename TOut>
void launch_cast(const TIn* in, TOut* out, long long n, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_cast<TIn, TOut><<<(unsigned)blocks, 256, 0, st>>>(in, out, n);
}

#define MFA_INST_S(T)                                                                                       \
  template void launch_frame_gather<T>(const LayoutDev&, const long long*, int, const T*, T*, cudaStream_t);     \
  template void launch_rhs_finalize<T>(const LayoutDev&, const long long*, const long long*, int, const T*,      \
                                       const T*, T*, cudaStream_t);                                              \
  template void launch_average<T>(const LayoutDev&, const long long*, const T*, T*, const T*, unsigned long long*, \
                                  cudaStream_t, int);                                                             \
  template void launch_decode_points<T>(const LayoutDev&, const double*, const double*, const double*, long long, \
                                        const int*, const T*, void*, int, cudaStream_t);                          \
  template void launch_cast<T, double>(const T*, double*, long long, cudaStream_t);                              \
  template void launch_cast<T, float>(const T*, float*, long long, cudaStream_t);

MFA_INST_S(double)
MFA_INST_S(float)
MFA_INST_S(ff)

}  // namespace mfa
