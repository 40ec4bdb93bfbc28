// Interface continuity metric (Sec. 2.2: C^0 .. C^{p-1} across subdomain
// interfaces; Algorithm 1 "check convergence metrics").  For a pair of
// subdomains that are neighbours along axis a, each local spline -- the L box
// of control points the subdomain used in its last solve: its own copy on U
// and, after a Schwarz step, the frame values it held (the lagged global
// iterate) -- is evaluated one-sidedly at the interface breakpoint with the
// host-built derivative rows, at every data point of the pair's common core
// along the other axes.  The block keeps the largest |left - right| per
// derivative order.  FP64 throughout (a diagnostic, not a data pass).
#include "mfa_internal.cuh"

namespace mfa {

namespace {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(ff v) { return (double)v.hi + (double)v.lo; }

constexpr int kJumpThreads = 128;

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kJumpThreads) k_interface_jumps(LayoutDev L, const long long* __restrict__ offL,
                                                                  const T* __restrict__ X,
                                                                  const T* __restrict__ Pprev, int use_frames,
                                                                  const JumpPair* __restrict__ pairs,
                                                                  const double* __restrict__ rows,
                                                                  const int* __restrict__ rowcp, int R,
                                                                  unsigned long long* out) {
  __shared__ double red[kJumpThreads / 32][MFA_MAX_DEGREE + 1];
  const JumpPair pr = pairs[blockIdx.x];
  const int a = pr.axis;
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;  // the other two axes, in order
  const int pa = L.ax[a].p, pb = L.ax[b].p, pc = L.ax[c].p;
  const long long nb = pr.k1[b] - pr.k0[b], nc = pr.k1[c] - pr.k0[c];
  const long long nsamp = nb * nc;
  double jmax[MFA_MAX_DEGREE + 1];
  for (int r = 0; r <= MFA_MAX_DEGREE; ++r) jmax[r] = 0.0;
  for (long long t = threadIdx.x; t < nsamp; t += blockDim.x) {
    const int kb = pr.k0[b] + (int)(t % nb), kc = pr.k0[c] + (int)(t / nb);
    const int gb0 = L.ax[b].span[kb], gc0 = L.ax[c].span[kc];
    const double* Nb = L.ax[b].vals_d + (long long)kb * (pb + 1);
    const double* Nc = L.ax[c].vals_d + (long long)kc * (pc + 1);
    double val[2][MFA_MAX_DEGREE + 1];
    for (int side = 0; side < 2; ++side) {
      const int sd = side ? pr.t : pr.s;
      int si[3];
      sub_pieces(L, sd, si[0], si[1], si[2]);
      const AxisSub sub[3] = {L.ax[0].subs[si[0]], L.ax[1].subs[si[1]], L.ax[2].subs[si[2]]};
      const int row = pr.iface + side;
      const int ga0 = rowcp[row];
      const double* D = rows + (long long)row * (R + 1) * (pa + 1);
      const long long off = offL[sd];
      const int nL0 = sub[0].nL, nL1 = sub[1].nL;
      for (int r = 0; r <= R; ++r) val[side][r] = 0.0;
      for (int ic = 0; ic <= pc; ++ic) {
        const double wc = Nc[ic];
        const int lc = gc0 + ic - sub[c].l0;
        if (wc == 0.0 || lc < 0 || lc >= sub[c].nL) continue;  // zero value past the box (window end)
        for (int ib = 0; ib <= pb; ++ib) {
          const double wb = Nb[ib];
          const int lb = gb0 + ib - sub[b].l0;
          if (wb == 0.0 || lb < 0 || lb >= sub[b].nL) continue;
          for (int ia = 0; ia <= pa; ++ia) {
            const int la = ga0 + ia - sub[a].l0;
            if (la < 0 || la >= sub[a].nL) continue;
            int l[3];
            l[a] = la;
            l[b] = lb;
            l[c] = lc;
            // owned copy on U; after a Schwarz step the frame held the lagged global iterate
            bool own = true;
            for (int x = 0; x < 3; ++x) own = own && l[x] >= sub[x].oU && l[x] < sub[x].oU + sub[x].nU;
            double v;
            if (own || !use_frames) {
              v = to_d(X[off + l[0] + (long long)nL0 * (l[1] + (long long)nL1 * l[2])]);
            } else {
              const long long g0 = sub[0].l0 + l[0], g1 = sub[1].l0 + l[1], g2 = sub[2].l0 + l[2];
              v = to_d(Pprev[g0 + L.ncp[0] * (g1 + L.ncp[1] * g2)]);
            }
            const double wv = wb * wc * v;
            for (int r = 0; r <= R; ++r) val[side][r] += D[r * (pa + 1) + ia] * wv;
          }
        }
      }
    }
    for (int r = 0; r <= R; ++r) jmax[r] = fmax(jmax[r], fabs(val[0][r] - val[1][r]));
  }
  // block maximum per order, then one atomic per order (non-negative doubles
  // order like their bit patterns)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = 0; r <= R; ++r) {
    double v = jmax[r];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) red[warp][r] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int r = 0; r <= R; ++r) {
      double v = 0.0;
      for (int w = 0; w < kJumpThreads / 32; ++w) v = fmax(v, red[w][r]);
      atomicMax(out + r, (unsigned long long)__double_as_longlong(v));
    }
  }
}

template <typename T>
void launch_interface_jumps(const LayoutDev& L, const long long* offL, const T* X, const T* Pprev, int use_frames,
                            const JumpPair* pairs, int npairs, const double* rows, const int* rowcp, int R,
                            unsigned long long* out, cudaStream_t st) {
  if (npairs <= 0) return;
  k_interface_jumps<T><<<npairs, kJumpThreads, 0, st>>>(L, offL, X, Pprev, use_frames, pairs, rows, rowcp, R, out);
}

template void launch_interface_jumps<double>(const LayoutDev&, const long long*, const double*, const double*, int,
                                             const JumpPair*, int, const double*, const int*, int,
                                             unsigned long long*, cudaStream_t);
template void launch_interface_jumps<ff>(const LayoutDev&, const long long*, const ff*, const ff*, int,
                                         const JumpPair*, int, const double*, const int*, int, unsigned long long*,
                                         cudaStream_t);

}  // namespace mfa
