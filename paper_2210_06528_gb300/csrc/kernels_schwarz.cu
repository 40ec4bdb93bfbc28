// Schwarz exchange and update kernels (Sec. 2.3.2, Algorithm 1 loop body) and
// scattered decode.
#include "mfa_internal.cuh"

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
  if (blocks > 152 * 16) blocks = 152 * 16;
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
    int j = (int)floor(u * ax.nspans);
    if (j > ax.nspans - 1) j = ax.nspans - 1;
    if (j < 0) j = 0;
    span[a] = j;
    basis_derivs(j, u, ax.p, ax.nspans, a < L.dim ? der[a] : 0, N[a]);
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

template <typename T>
void launch_decode_points(const LayoutDev& L, const double* lo, const double* hi, const double* pts, long long npts,
                          const int* deriv, const T* P, void* out, int out_dtype, cudaStream_t st) {
  long long blocks = (npts + 127) / 128;
  k_decode_points<T><<<(unsigned)blocks, 128, 0, st>>>(L, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], pts, npts,
                                                       deriv[0], deriv[1], deriv[2], P, out, out_dtype);
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

template <typename T>
void launch_decode_points_inst(const InstDesc* desc, const int* qinst, const long long* pt_off, int nq,
                               long long npts, const double* pts, const T* P, double* out, cudaStream_t st) {
  if (npts <= 0 || nq <= 0) return;
  k_decode_points_inst<T><<<(unsigned)((npts + 127) / 128), 128, 0, st>>>(desc, qinst, pt_off, nq, pts, P, out);
}

template void launch_decode_points_inst<double>(const InstDesc*, const int*, const long long*, int, long long,
                                                const double*, const double*, double*, cudaStream_t);
template void launch_decode_points_inst<ff>(const InstDesc*, const int*, const long long*, int, long long,
                                            const double*, const ff*, double*, cudaStream_t);

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
