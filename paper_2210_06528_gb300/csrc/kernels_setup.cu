// Setup kernels (Algorithm 1 "Setup"): Cox-de Boor basis tables, banded
// per-axis Gram matrices of every subdomain window and their Cholesky factors.
// All three are tiny (per-axis work, O(M_a p^2)); they run in FP64.
#include "mfa_internal.cuh"

namespace mfa {

// Knot t_i of the clamped uniform knot vector with `nspans` spans, degree p.
__device__ __forceinline__ double knot_at(int i, int p, int nspans) {
  if (i <= p) return 0.0;
  if (i >= nspans + p) return 1.0;
  return (double)(i - p) / (double)nspans;
}

// Basis values N_{j+r,p}(u), r = 0..p, on knot span j (global span index) by
// the Cox-de Boor recurrence (Sec. 2.1, Eq. nurbs-basis with W = 1), raising
// the degree from 0 to p on the p+1 functions that are nonzero on the span.
// Writing i = j + p for the knot index of the span's left end, degree q keeps
// Nq[r] = N_{i-q+r,q} for r = 0..q and
//   Nq[r] = (u - t_{i-q+r}) / (t_{i+r} - t_{i-q+r}) * N_{q-1}[r-1]
//         + (t_{i+r+1} - u) / (t_{i+r+1} - t_{i-q+r+1}) * N_{q-1}[r].
// Both denominators are positive on a non-empty span.
__device__ void cox_de_boor(int j, double u, int p, int nspans, double* N) {
  const int i = j + p;
  N[0] = 1.0;
  for (int q = 1; q <= p; ++q) {
    double carry = 0.0;  // contribution of N_{q-1}[r-1] to Nq[r]
    for (int r = 0; r < q; ++r) {
      const double tl = knot_at(i - q + r + 1, p, nspans);
      const double tr = knot_at(i + r + 1, p, nspans);
      const double w = N[r] / (tr - tl);
      const double right = (tr - u) * w;            // N_{q-1}[r] -> Nq[r]
      const double left_next = (u - tl) * w;        // N_{q-1}[r] -> Nq[r+1]
      N[r] = carry + right;
      carry = left_next;
    }
    N[q] = carry;
  }
}

__global__ void k_basis(int M, int nspans, int p, int* span, double* vd, float* vf, ff* vff) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  // span index: largest j with j/nspans <= k/(M-1), exact in integers
  int j = 0;
  double u = 0.0;
  if (M > 1) {
    long long num = (long long)k * nspans;
    j = (int)(num / (M - 1));
    if (j > nspans - 1) j = nspans - 1;
    u = (double)k / (double)(M - 1);
  }
  double N[MFA_MAX_DEGREE + 1];
  cox_de_boor(j, u, p, nspans, N);
  span[k] = j;
  for (int r = 0; r <= p; ++r) {
    vd[(long long)k * (p + 1) + r] = N[r];
    vf[(long long)k * (p + 1) + r] = (float)N[r];
    if (vff) vff[(long long)k * (p + 1) + r] = ff(N[r]);
  }
}

void launch_basis(const AxisDev& ax, int* span, double* vd, float* vf, ff* vff, cudaStream_t st) {
  int threads = 128;
  int blocks = (ax.M + threads - 1) / threads;
  k_basis<<<blocks, threads, 0, st>>>(ax.M, ax.nspans, ax.p, span, vd, vf, vff);
}

// Gram band of one window: A_L = N_L^T N_L summed over the window's points
// (the normal matrix of Eq. minimization-problem along one axis).  Each data
// point touches the p+1 control points of its span; the point sitting on the
// window's closing breakpoint has a zero last value whose index lies past L
// and is skipped.  One thread per piece; serial FP64 sums.
__global__ void k_gram(AxisDev ax, double* AL) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ax.S) return;
  const AxisSub sb = ax.subs[s];
  const int p = ax.p, w = p + 1;
  double* A = AL + (long long)sb.bandL * w;
  for (int i = 0; i < sb.nL * w; ++i) A[i] = 0.0;
  for (int k = sb.k0; k < sb.k0 + sb.m; ++k) {
    const int j = ax.span[k];
    const double* v = ax.vals_d + (long long)k * w;
    for (int r = 0; r <= p; ++r) {
      const int l = j + r - sb.l0;
      if (l < 0 || l >= sb.nL) continue;
      for (int r2 = r; r2 <= p; ++r2) {
        const int l2 = j + r2 - sb.l0;
        if (l2 >= sb.nL) continue;
        A[l * w + (r2 - r)] += v[r] * v[r2];
      }
    }
  }
}

void launch_gram(const AxisDev& ax, double* AL, cudaStream_t st) {
  k_gram<<<(ax.S + 63) / 64, 64, 0, st>>>(ax, AL);
}

// Banded Cholesky A = L L^T of the n x n principal block of A_L starting at
// row `o` (Sec. 2.3.1: Cholesky on the normal equations).  Row-oriented:
//   L(i,j) = (A(j,i) - sum_{k<j} L(i,k) L(j,k)) / L(j,j),  i-p <= j < i
//   L(i,i) = sqrt(A(i,i) - sum_{k<i} L(i,k)^2).
// A pivot that is not positive, or falls below 1e-13 of its diagonal entry,
// marks the status word MFA_ERR_NOT_SPD and the factor is left unusable.
__device__ void band_cholesky(const double* A, int o, int n, int p, double* F, float* Ff, ff* Fff, int* status) {
  const int w = p + 1;
  for (int i = 0; i < n; ++i) {
    for (int e = p; e >= 1; --e) {
      const int j = i - e;
      if (j < 0) continue;
      double s = A[(long long)(o + j) * w + e];
      for (int f = e + 1; f <= p; ++f) {
        if (i - f < 0) continue;
        s -= F[i * w + f] * F[j * w + (f - e)];
      }
      F[i * w + e] = s * F[j * w];
    }
    const double aii = A[(long long)(o + i) * w];
    double dsum = aii;
    for (int e = 1; e <= p; ++e)
      if (i - e >= 0) dsum -= F[i * w + e] * F[i * w + e];
    if (!(dsum > 1e-13 * aii) || !(aii > 0.0)) {
      atomicExch(status, MFA_ERR_NOT_SPD);
      dsum = 1.0;
    }
    F[i * w] = 1.0 / sqrt(dsum);
  }
  for (int i = 0; i < n * w; ++i) {
    Ff[i] = (float)F[i];
    Fff[i] = ff(F[i]);
  }
}

__global__ void k_chol(AxisDev ax, const double* AL, double* fLd, float* fLf, ff* fLff, double* fUd, float* fUf,
                       ff* fUff, int* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * ax.S) return;
  const int s = t >> 1;
  const AxisSub sb = ax.subs[s];
  const int w = ax.p + 1;
  const double* A = AL + (long long)sb.bandL * w;
  if ((t & 1) == 0)
    band_cholesky(A, 0, sb.nL, ax.p, fLd + (long long)sb.bandL * w, fLf + (long long)sb.bandL * w,
                  fLff + (long long)sb.bandL * w, status);
  else
    band_cholesky(A, sb.oU, sb.nU, ax.p, fUd + (long long)sb.bandU * w, fUf + (long long)sb.bandU * w,
                  fUff + (long long)sb.bandU * w, status);
}

void launch_chol(const AxisDev& ax, const double* AL, double* fLd, float* fLf, ff* fLff, double* fUd, float* fUf,
                 ff* fUff, int* status, cudaStream_t st) {
  int n = 2 * ax.S;
  k_chol<<<(n + 63) / 64, 64, 0, st>>>(ax, AL, fLd, fLf, fLff, fUd, fUf, fUff, status);
}

}  // namespace mfa

namespace mfa {

// ---------------------------------------------------------------------------
// Batched setup: one launch evaluates the basis of every axis; one launch
// assembles the Gram band of every piece of every axis (one CTA per piece,
// one thread per band entry) and factors it in shared memory.
// ---------------------------------------------------------------------------

struct SetupArgs {
  AxisDev ax[3];
  int naxes;
  int* span[3];
  double* vd[3];
  float* vf[3];
  ff* vff[3];
  double* AL[3];
  double *fLd[3], *fUd[3];
  float *fLf[3], *fUf[3];
  ff *fLff[3], *fUff[3];
};

__global__ void k_basis_all(SetupArgs A) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int a = 0;
  while (a < A.naxes && k >= A.ax[a].M) {
    k -= A.ax[a].M;
    ++a;
  }
  if (a >= A.naxes) return;
  const AxisDev& ax = A.ax[a];
  const int p = ax.p;
  int M = ax.M, nspans = ax.nspans, kl = k, j0 = 0;
  int j = 0;
  double u = 0.0;
  if (ax.kmode == KMODE_CLAMPED) {
    // clamped interfaces: the point's span on the grid (largest j with
    // j/gspans <= k/(M-1), exact in integers), the core [a, b) holding it, and
    // that core's own clamped uniform knots of b - a spans at the local
    // parameter (x - a)/(b - a), x = u * gspans; spans numbered from the
    // core's first owned control point
    const int gs = ax.gspans;
    int jg = 0;
    double x = 0.0;
    if (M > 1) {
      jg = (int)(((long long)k * gs) / (M - 1));
      if (jg > gs - 1) jg = gs - 1;
      x = (double)k * (double)gs / (double)(M - 1);
    }
    int lo = 0, hi = ax.S - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ax.subs[mid].a <= jg) lo = mid;
      else hi = mid - 1;
    }
    const AxisSub sb = ax.subs[lo];
    nspans = sb.b - sb.a;
    j = jg - sb.a;
    u = (x - (double)sb.a) / (double)nspans;
    j0 = sb.l0 + sb.oU;
  } else {
    if (ax.pieces) {
      // independent fits side by side: find the piece holding point k (pieces
      // are sorted by k0), then use its own knot vector and parameters
      int lo = 0, hi = ax.S - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ax.subs[mid].k0 <= k) lo = mid;
        else hi = mid - 1;
      }
      const AxisSub sb = ax.subs[lo];
      M = sb.m;
      nspans = sb.w1 - sb.w0;
      kl = k - sb.k0;
      j0 = sb.l0;
    }
    if (M > 1) {
      j = (int)(((long long)kl * nspans) / (M - 1));
      if (j > nspans - 1) j = nspans - 1;
      u = (double)kl / (double)(M - 1);
    }
  }
  double N[MFA_MAX_DEGREE + 1];
  cox_de_boor(j, u, p, nspans, N);
  if (ax.wts) {
    // rational basis R_g = N_g W_g / sum_h N_h W_h (Eq. nurbs-basis)
    double wsum = 0.0;
    for (int r = 0; r <= p; ++r) {
      N[r] *= ax.wts[j0 + j + r];
      wsum += N[r];
    }
    for (int r = 0; r <= p; ++r) N[r] /= wsum;
  }
  A.span[a][k] = j0 + j;
  for (int r = 0; r <= p; ++r) {
    A.vd[a][(long long)k * (p + 1) + r] = N[r];
    A.vf[a][(long long)k * (p + 1) + r] = (float)N[r];
    A.vff[a][(long long)k * (p + 1) + r] = ff(N[r]);
  }
}

// Banded Cholesky of the n x n block of A (upper band storage, row stride w)
// starting at row o; writes the factor (1/L(i,i) at [i*w], L(i,i-e) at
// [i*w+e]) in FP64, FP32 and float-float.  Same recurrence as band_cholesky.
__device__ void band_cholesky_smem(const double* A, int o, int n, int p, double* F, double* Fd, float* Ff, ff* Fff,
                                   int* status) {
  const int w = p + 1;
  for (int i = 0; i < n; ++i) {
    for (int e = p; e >= 1; --e) {
      const int j = i - e;
      if (j < 0) continue;
      double s = A[(o + j) * w + e];
      for (int f = e + 1; f <= p; ++f) {
        if (i - f < 0) continue;
        s -= F[i * w + f] * F[j * w + (f - e)];
      }
      F[i * w + e] = s * F[j * w];
    }
    const double aii = A[(o + i) * w];
    double dsum = aii;
    for (int e = 1; e <= p; ++e)
      if (i - e >= 0) dsum -= F[i * w + e] * F[i * w + e];
    if (!(dsum > 1e-13 * aii) || !(aii > 0.0)) {
      atomicExch(status, MFA_ERR_NOT_SPD);
      dsum = 1.0;
    }
    F[i * w] = 1.0 / sqrt(dsum);
  }
  for (int i = 0; i < n * w; ++i) {
    Fd[i] = F[i];
    Ff[i] = (float)F[i];
    Fff[i] = ff(F[i]);
  }
}

__global__ void k_gram_chol_all(SetupArgs A, int* status) {
  extern __shared__ double sh[];
  int b = blockIdx.x, a = 0;
  while (a < A.naxes && b >= A.ax[a].S) {
    b -= A.ax[a].S;
    ++a;
  }
  if (a >= A.naxes) return;
  const AxisDev& ax = A.ax[a];
  const AxisSub sb = ax.subs[b];
  const int p = ax.p, w = p + 1, nL = sb.nL;
  double* As = sh;            // [nL][w]
  double* F = sh + nL * w;    // [nL][w] scratch factor
  // A(l, l+e) = sum over window points of N_g N_{g+e}, g = l0 + l, on spans [g+e-p, g]
  for (int t = threadIdx.x; t < nL * w; t += blockDim.x) {
    const int l = t / w, e = t - l * w;
    const int g = sb.l0 + l;
    double acc = 0.0;
    if (l + e < nL) {
      const int jlo = max(g + e - p, 0), jhi = min(g, ax.nspans - 1);
      if (jlo <= jhi) {
        int kb = ax.span_start[jlo], ke = ax.span_start[jhi + 1];
        kb = max(kb, sb.k0);
        ke = min(ke, sb.k0 + sb.m);
        for (int k = kb; k < ke; ++k) {
          const int r = g - ax.span[k];
          const double* v = A.vd[a] + (long long)k * w;
          acc += v[r] * v[r + e];
        }
      }
    }
    As[t] = acc;
    A.AL[a][(long long)sb.bandL * w + t] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    band_cholesky_smem(As, 0, nL, p, F, A.fLd[a] + (long long)sb.bandL * w, A.fLf[a] + (long long)sb.bandL * w,
                       A.fLff[a] + (long long)sb.bandL * w, status);
  } else if (threadIdx.x == 32) {
    // the owned block needs its own scratch: reuse the upper half of F's space
    double* FU = F + (size_t)nL * w;
    band_cholesky_smem(As, sb.oU, sb.nU, p, FU, A.fUd[a] + (long long)sb.bandU * w, A.fUf[a] + (long long)sb.bandU * w,
                       A.fUff[a] + (long long)sb.bandU * w, status);
  }
}

void launch_setup_all(const AxisDev* ax, int naxes, int maxnL, int* status, cudaStream_t st) {
  SetupArgs A{};
  A.naxes = naxes;
  int totalM = 0, totalS = 0, maxw = 1;
  for (int a = 0; a < naxes; ++a) {
    A.ax[a] = ax[a];
    A.span[a] = const_cast<int*>(ax[a].span);
    A.vd[a] = const_cast<double*>(ax[a].vals_d);
    A.vf[a] = const_cast<float*>(ax[a].vals_f);
    A.vff[a] = const_cast<ff*>(ax[a].vals_ff);
    A.AL[a] = const_cast<double*>(ax[a].AL);
    A.fLd[a] = const_cast<double*>(ax[a].facL_d);
    A.fLf[a] = const_cast<float*>(ax[a].facL_f);
    A.fLff[a] = const_cast<ff*>(ax[a].facL_ff);
    A.fUd[a] = const_cast<double*>(ax[a].facU_d);
    A.fUf[a] = const_cast<float*>(ax[a].facU_f);
    A.fUff[a] = const_cast<ff*>(ax[a].facU_ff);
    totalM += ax[a].M;
    totalS += ax[a].S;
    maxw = ax[a].p + 1 > maxw ? ax[a].p + 1 : maxw;
  }
  k_basis_all<<<(totalM + 127) / 128, 128, 0, st>>>(A);
  // shared: Gram band, L-factor and U-factor scratch of the largest piece
  const size_t smem = (size_t)3 * maxnL * maxw * sizeof(double);
  k_gram_chol_all<<<totalS, 128, smem, st>>>(A, status);
}

}  // namespace mfa
