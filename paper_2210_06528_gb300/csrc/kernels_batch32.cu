// FP32 data passes of a batch of independent fits (MFA_PREC_FP32): FP32 basis
// values, N^T Q and decode; FP64 Gram matrices and Cholesky factors, banded
// solves in float-float with the factors' float-float copies.
//
// One CTA per item (rows of one instance).  The CTA loads the instance's x
// basis values (padded to W per point) and span starts into shared memory
// once; then every warp works through its own rows with warp-level
// synchronisation only (3-D: whole planes per warp; 2-D: the rows of a range
// of y knot spans).  A warp streams its rows in chunks of at most kB32Stage
// values (rows padded to an odd pitch), double-buffered: the next chunk is
// copied asynchronously (cp.async) while the current one is computed:
//  - x: one lane per (row, segment of knot spans) walks the segment's points
//    left to right with p + 1 register accumulators; a control point is
//    stored when its last span has passed.  A control point whose support
//    straddles two segments gets the later segment's part first and the
//    earlier segment's part is added afterwards, in that fixed order.
//  - y, whole planes in a chunk: one lane per (plane, y control point, x
//    control point) sums the rows of its support.  Rows of a larger plane:
//    one lane per x control point carries the p + 1 y control points still
//    open (registers, or shared memory between chunks when n0 > 32) and
//    emits each one when no later row touches it.  Where warps split a 2-D
//    instance, the control points of a boundary get the earlier warp's part
//    plus the later warp's part, added after a CTA barrier.
//  2-D and 1-D instances are then complete (right-hand sides, as float-float
//  for the solves); 3-D instances write their xy-reduced planes and a second
//  kernel contracts z.
//  Refinement projects r = q - (N P32) instead of q, P32 the FP32 copy of
//  the control points: per chunk the y-expanded control points of its rows
//  (from the z-expanded planes DZ of a 3-D instance, which k_b32_zexpand
//  writes beforehand), then every lane decodes its points in the same walk
//  (one step of iterative refinement; its rounding is relative to |r|).
//
// Residual.  The same walk with the decode only: E = q - value, sum of E^2
// and max |E| per lane (FP32), per warp and CTA in FP64 in fixed order.
#include "mfa_internal.cuh"

namespace mfa {

namespace {

constexpr int kPF = kB32Stage / 32;  // staged values per lane and chunk

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
// 4-byte asynchronous copy global -> shared, issued only where ok != 0
__device__ __forceinline__ void cp_async4(unsigned dst, const float* src, int ok) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.ca.shared.global [%0], [%1], 4;\n}\n" ::"r"(dst),
      "l"(src), "r"(ok)
      : "memory");
}
// Shared-memory loads at 32-bit shared addresses.
__device__ __forceinline__ float lds(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds4(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__host__ __device__ constexpr int r4(int x) { return (x + 3) & ~3; }

// floor(e / d) for e * d < 2^32 with mg = ceil(2^32 / d): the product
// e * mg / 2^32 exceeds e / d by less than e / 2^32 < 1 / d, which never
// carries past the next integer; d = 1 is taken apart (mg would need 33 bits).
// ceil(2^32 / d) = floor((2^32 - 1) / d) + 1 for d >= 2 (32-bit division).
__device__ __forceinline__ unsigned fdiv(unsigned e, unsigned d, unsigned mg) {
  return d == 1 ? e : __umulhi(e, mg);
}
__device__ __forceinline__ unsigned fmagic(unsigned d) { return d <= 1 ? 0u : 0xffffffffu / d + 1u; }

// Floats of one warp's shared-memory region (each part a multiple of 4).
__host__ __device__ inline int b32_warp_floats(const B32Caps& c, int mode) {
  int f = 2 * r4(c.stage);  // staged rows, two buffers
  if (mode != B32_RESIDUAL) f += r4(c.xr) + r4(c.ring);
  if (mode != B32_PROJECT) f += r4(c.xr);
  return f;
}
// Floats of the CTA's tables: x basis values (W per point), x span starts, y
// span starts, y basis values (W per row) and the y span of every row.
__host__ __device__ inline int b32_cta_floats(const B32Caps& c) {
  return r4(c.vb) + r4(c.sx) + r4(c.sy) + r4(c.vy) + r4(c.ysp);
}

struct B32Warp {
  float* stage;  // two buffers of the launch's stage capacity
  float* xr;     // [row of the chunk][n0 | 1]: x-reduced rows
  float* ring;   // streamed planes with n0 > 32: open y control points between chunks
  float* dzy;    // [row of the chunk][n0 | 1]: z- and y-expanded control points
};

struct B32Tables {
  const float* vb;  // [M0][W] x basis values
  const int* sx;    // [ns0 + 1] first point of every x span
  const int* sy;    // [ns1 + 1] first row of every y span
  const float* vy;  // [M1][W] y basis values
  const int* ysp;   // [M1] y span of every row
};

// A warp's rows [ra, rb) of one instance (2-D: the rows of y spans [sa, sb)).
template <int P, int MODE>
__device__ __forceinline__ void b32_warp(const B32Inst& D, const B32Item& it, const B32Warp& L, const B32Tables& T,
                                         int w, int ra, int rb, int sa, int sb, int cap_stage,
                                         const float* __restrict__ Q, const float* __restrict__ P32,
                                         const float* __restrict__ DZ, ff* __restrict__ X, float* __restrict__ R,
                                         float* __restrict__ Z, float& s2, float& emax) {
  constexpr int W = P < 4 ? 4 : 8;  // basis values per point / row in shared memory (padded)
  const int lane = threadIdx.x & 31;
  const int M0 = D.M[0], M1 = D.M[1], n0 = D.n[0], n1 = D.n[1];
  const int py = D.dim >= 2 ? P : 0;
  const int ns0 = n0 - P, ns1 = n1 - py;
  const int pitch = M0 | 1, pad = pitch - M0, n0s = n0 | 1;
  const unsigned mg0 = fmagic(M0), mg1 = fmagic(M1), mgn0 = fmagic(n0);
  int rc_mg = 0;  // rows of the chunk whose magic number is in mgh
  unsigned mgh = 0;
  const int S = D.S;
  const unsigned mgS = fmagic(S);
  const bool whole = D.mode == 0;
  const int plane_cp = n1 * n0;
  // control points the decode expands along y: the instance's own (2-D), or
  // its z-expanded planes (3-D)
  const float* Pi = MODE == B32_PROJECT ? nullptr : D.dim == 3 ? DZ + D.r_off : P32 + D.x_off;

  int row = ra;
  int k2 = row / M1, k1 = row - k2 * M1;
  auto rows_at = [&](int r, int kk1) { return whole ? min(D.np * M1, rb - r) : min(D.R, min(M1 - kk1, rb - r)); };
  // rows [r, r + rc) into stage buffer bf, value e = i M0 + k at i * pitch + k
  const int scap = r4(cap_stage);
  auto load = [&](int r, int rc, int bf) {
    const float* src = Q + D.q_off + (long long)r * M0 + lane;
    const unsigned dst = smem_u32(L.stage + bf * scap);
    const int n = rc * M0;
#pragma unroll
    for (int m = 0; m < kPF; ++m) {
      const unsigned e = lane + 32 * m;
      cp_async4(dst + 4u * (e + __umulhi(e, mg0) * pad), src + 32 * m, (int)e < n);
    }
    cp_async_commit();
  };
  // y emission: 3-D xy-reduced planes; 2-D control points, or the partial
  // sums at this warp's boundary spans sa / sb when warps split the instance
  // (descriptor fields in registers: D lives in shared memory, and stores
  // through these pointers would otherwise make every emission reload it)
  const int dim = D.dim;
  float* const Rb = dim == 3 ? R + D.r_off : nullptr;
  float* const Zb = dim == 2 ? Z + it.z_off : nullptr;
  ff* const Xb = MODE != B32_RESIDUAL ? X + D.x_off : nullptr;
  auto emit = [=](int kk2, int j1, int j0, float v) {
    if (dim == 3) {
      Rb[((long long)kk2 * n1 + j1) * n0 + j0] = v;
    } else if (sa > 0 && j1 < sa + P) {
      Zb[(2 * w * P + (j1 - sa)) * n0 + j0] = v;
    } else if (sb < ns1 && j1 >= sb) {
      Zb[((2 * w + 1) * P + (j1 - sb)) * n0 + j0] = v;
    } else {
      Xb[(long long)j1 * n0 + j0] = ff(v);
    }
  };
  auto yvals = [&](int kk1, float* v) {
    const float4 v0 = *reinterpret_cast<const float4*>(T.vy + kk1 * W);
    v[0] = v0.x;
    v[1] = v0.y;
    v[2] = v0.z;
    v[3] = v0.w;
    if (W == 8) {
      const float4 v1 = *reinterpret_cast<const float4*>(T.vy + kk1 * W + 4);
      v[4 % W] = v1.x;
      v[5 % W] = v1.y;
      v[6 % W] = v1.z;
      v[7 % W] = v1.w;
    }
  };

  int rc = rows_at(row, k1);
  int buf = 0;
  load(row, rc, 0);
  // streamed planes: the open y control points [cur, cur + P]
  int cur = sa;
  bool fresh = true;
  float ay[P + 1];
#pragma unroll
  for (int c = 0; c <= P; ++c) ay[c] = 0.f;

  while (row < rb) {
    const float* stage = L.stage + buf * scap;
    const int nrow = row + rc;
    int nk1 = k1 + rc, nk2 = k2;
    if (whole) {
      nk1 = 0;
      nk2 = k2 + (int)fdiv(rc, M1, mg1);
    } else if (nk1 == M1) {
      nk1 = 0;
      nk2 = k2 + 1;
    }
    const int nrc = nrow < rb ? rows_at(nrow, nk1) : 0;
    if (nrc) {
      load(nrow, nrc, buf ^ 1);  // in flight during this chunk's arithmetic
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    if (MODE != B32_PROJECT) {
      // z- and y-expanded control points of the chunk's rows, K per lane at a
      // time: their loads (from L2) all in flight before the first sum
      constexpr int K = P <= 3 ? 4 : 2;
      const int ne = rc * n0;
      for (int t0 = 0; t0 < ne; t0 += 32 * K) {
        float g[K][P + 1];
        int kk[K], at[K];
#pragma unroll
        for (int u = 0; u < K; ++u) {
          const int t = min(t0 + 32 * u + lane, ne - 1);
          const int rr = (int)fdiv(t, n0, mgn0), j0 = t - rr * n0;
          const int pl = whole ? (int)fdiv(rr, M1, mg1) : 0;
          kk[u] = whole ? rr - pl * M1 : k1 + rr;
          at[u] = rr * n0s + j0;
          const float* src = (D.dim == 3 ? Pi + (long long)(k2 + pl) * plane_cp : Pi) + T.ysp[kk[u]] * n0 + j0;
#pragma unroll
          for (int c = 0; c <= P; ++c) g[u][c] = c <= py ? __ldg(src + c * n0) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < K; ++u) {
          const float* v = T.vy + kk[u] * W;
          float a = 0.f;
#pragma unroll
          for (int c = 0; c <= P; ++c)
            if (c <= py) a = fmaf(v[c], g[u][c], a);
          if (t0 + 32 * u + lane < ne) L.dzy[at[u]] = a;
        }
      }
      __syncwarp();
    }
    // x: one lane per (pair of rows i and i + H, segment)
    {
      const int H = (rc + 1) >> 1;
      if (H != rc_mg) {
        rc_mg = H;
        mgh = fmagic(H);
      }
      const int tasks = H * S;
      bool have_left = false, left2 = false;
      float la[P], lb[P];
      int lpa = 0, lpb = 0;
      for (int t = lane; t < tasks; t += 32) {
        const int g = (int)fdiv(t, H, mgh), ia = t - g * H;
        const bool two = ia + H < rc;
        const int ib = two ? ia + H : ia;
        const int ga = (int)fdiv(ns0 * g, S, mgS), gb = (int)fdiv(ns0 * (g + 1), S, mgS);
        const float* pa = stage + ia * pitch;
        const float* pb = stage + ib * pitch;
        float* xa = MODE != B32_RESIDUAL ? L.xr + ia * n0s : nullptr;
        float* xb = MODE != B32_RESIDUAL ? L.xr + ib * n0s : nullptr;
        const float* dra = MODE != B32_PROJECT ? L.dzy + ia * n0s : nullptr;
        const float* drb = MODE != B32_PROJECT ? L.dzy + ib * n0s : nullptr;
        const float m2 = two ? 1.f : 0.f;  // residual: row b counted once
        // accumulators of rows a and b side by side: paired FP32 instructions
        // (per lane the same rounding as fmaf)
        float2 acc[P + 1];
#pragma unroll
        for (int c = 0; c <= P; ++c) acc[c] = make_float2(0.f, 0.f);
        int k = T.sx[ga];
        // 32-bit shared addresses of point k of rows a and b and of its basis values
        unsigned qa_at = smem_u32(pa) + 4u * k;
        const unsigned qb_off = smem_u32(pb) - smem_u32(pa);
        unsigned b_at = smem_u32(T.vb) + 4u * W * k;
        for (int s = ga; s < gb; ++s) {
          const int ke = T.sx[s + 1];
          float2 d2[P + 1];
          if (MODE != B32_PROJECT) {
#pragma unroll
            for (int c = 0; c <= P; ++c) d2[c] = make_float2(dra[s + c], drb[s + c]);
          }
          for (; k < ke; ++k, qa_at += 4u, b_at += 4u * W) {
            float qa = lds(qa_at), qb = lds(qa_at + qb_off);
            float b[W];
            const float4 b0 = lds4(b_at);
            b[0] = b0.x;
            b[1] = b0.y;
            b[2] = b0.z;
            b[3] = b0.w;
            if (W == 8) {
              const float4 b1 = lds4(b_at + 16u);
              b[4 % W] = b1.x;
              b[5 % W] = b1.y;
              b[6 % W] = b1.z;
              b[7 % W] = b1.w;
            }
            if (MODE != B32_PROJECT) {
              float2 v2 = make_float2(0.f, 0.f);
#pragma unroll
              for (int c = 0; c <= P; ++c) v2 = __ffma2_rn(make_float2(b[c], b[c]), d2[c], v2);
              qa -= v2.x;
              qb -= v2.y;
              if (MODE == B32_RESIDUAL) {
                const float eb = qb * m2;
                s2 = fmaf(qa, qa, s2);
                s2 = fmaf(eb, eb, s2);
                emax = fmaxf(emax, fmaxf(fabsf(qa), fabsf(eb)));
              }
            }
            if (MODE != B32_RESIDUAL) {
              const float2 q2 = make_float2(qa, qb);
#pragma unroll
              for (int c = 0; c <= P; ++c) acc[c] = __ffma2_rn(make_float2(b[c], b[c]), q2, acc[c]);
            }
          }
          if (MODE != B32_RESIDUAL) {
            // complete, or this segment's part of a straddling control point
            xa[s] = acc[0].x;
            if (two) xb[s] = acc[0].y;
#pragma unroll
            for (int c = 0; c < P; ++c) acc[c] = acc[c + 1];
            acc[P] = make_float2(0.f, 0.f);
          }
        }
        if (MODE != B32_RESIDUAL) {
          if (gb == ns0) {
#pragma unroll
            for (int c = 0; c < P; ++c) {
              xa[ns0 + c] = acc[c].x;
              if (two) xb[ns0 + c] = acc[c].y;
            }
          } else {  // S > 1: one task per lane (row pairs x S <= 32)
            have_left = true;
            left2 = two;
#pragma unroll
            for (int c = 0; c < P; ++c) {
              la[c] = acc[c].x;
              lb[c] = acc[c].y;
            }
            lpa = ia * n0s + gb;
            lpb = ib * n0s + gb;
          }
        }
      }
      if (MODE != B32_RESIDUAL) {
        __syncwarp();
        if (have_left) {
#pragma unroll
          for (int c = 0; c < P; ++c) {
            L.xr[lpa + c] += la[c];
            if (left2) L.xr[lpb + c] += lb[c];
          }
        }
        __syncwarp();
      }
    }
    if (MODE != B32_RESIDUAL) {
      if (D.dim == 1) {
        for (int j0 = lane; j0 < n0; j0 += 32) X[D.x_off + j0] = ff(L.xr[j0]);
      } else if (whole) {
        // whole planes: one lane per (plane, x control point) walks the
        // plane's rows with the p + 1 open y control points in registers
        const int npl = (int)fdiv(rc, M1, mg1);
        const int tasks = npl * n0;
        for (int t0 = 0; t0 < tasks; t0 += 32) {
          const int t = t0 + lane;
          const bool ok = t < tasks;
          const int pl = ok ? (int)fdiv(t, n0, mgn0) : 0;
          const int j0 = ok ? t - pl * n0 : 0;
          const float* xc = L.xr + pl * M1 * n0s + j0;
          float a[P + 1];
#pragma unroll
          for (int c = 0; c <= P; ++c) a[c] = 0.f;
          int cc = 0;
          for (int kk = 0; kk < M1;) {
            // the rows of span sr, after the control points before it are emitted
            const int sr = T.ysp[kk];
            while (cc < sr) {
              if (ok) emit(k2 + pl, cc, j0, a[0]);
#pragma unroll
              for (int c = 0; c < P; ++c) a[c] = a[c + 1];
              a[P] = 0.f;
              ++cc;
            }
            const int ke = max(kk + 1, T.sy[sr + 1]);
#pragma unroll 2
            for (; kk < ke; ++kk) {
              const float x = xc[kk * n0s];
              float v[W];
              yvals(kk, v);
#pragma unroll
              for (int c = 0; c <= P; ++c) a[c] = fmaf(v[c], x, a[c]);
            }
          }
          if (ok) {
#pragma unroll
            for (int c = 0; c <= P; ++c) emit(k2 + pl, cc + c, j0, a[c]);
          }
        }
      } else {
        // streamed plane: open y control points [cur, cur + P] per x control point
        const int NC = (n0 + 31) >> 5;
        const bool pend = (k1 + rc == M1) || (nrow == rb);
        int cc = cur;
        for (int m = 0; m < NC; ++m) {
          const int j0 = lane + 32 * m;
          const bool ok = j0 < n0;
          float a[P + 1];
#pragma unroll
          for (int c = 0; c <= P; ++c)
            a[c] = NC == 1 ? ay[c] : (fresh ? 0.f : L.ring[(m * (P + 1) + c) * 32 + lane]);
          cc = cur;
          for (int rr = 0; rr < rc;) {
            const int sr = T.ysp[k1 + rr];
            while (cc < sr) {
              if (ok) emit(k2, cc, j0, a[0]);
#pragma unroll
              for (int c = 0; c < P; ++c) a[c] = a[c + 1];
              a[P] = 0.f;
              ++cc;
            }
            const int re = min(rc, max(rr + 1, T.sy[sr + 1] - k1));
#pragma unroll 2
            for (; rr < re; ++rr) {
              const float x = ok ? L.xr[rr * n0s + j0] : 0.f;
              float v[W];
              yvals(k1 + rr, v);
#pragma unroll
              for (int c = 0; c <= P; ++c) a[c] = fmaf(v[c], x, a[c]);
            }
          }
          if (pend) {
#pragma unroll
            for (int c = 0; c <= P; ++c) {
              if (ok) emit(k2, cc + c, j0, a[c]);
              a[c] = 0.f;
            }
          }
          if (NC == 1) {
#pragma unroll
            for (int c = 0; c <= P; ++c) ay[c] = a[c];
          } else if (!pend) {
#pragma unroll
            for (int c = 0; c <= P; ++c) L.ring[(m * (P + 1) + c) * 32 + lane] = a[c];
          }
        }
        fresh = pend;
        cur = pend ? 0 : cc;
      }
    }
    __syncwarp();  // the staged rows and x-reduced rows are free again
    row = nrow;
    k1 = nk1;
    k2 = nk2;
    rc = nrc;
    buf ^= 1;
  }
}

// (refinement at degree >= 6 needs well over 128 registers: one CTA per SM)
template <int P, int MODE>
__global__ void __launch_bounds__(kB32Threads, MODE == B32_REFINE && P >= 6 ? 1 : 2)
    k_b32(const B32Inst* __restrict__ insts, const B32Item* __restrict__ items, int base, B32Caps cap,
          const float* __restrict__ Q, const float* __restrict__ P32, const float* __restrict__ DZ,
          ff* __restrict__ X, float* __restrict__ R, float* __restrict__ Z, double* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  __shared__ double red[kB32Threads / 32][2];
  __shared__ B32Inst Ds;
  __shared__ B32Item its;
  constexpr int W = P < 4 ? 4 : 8;
  if (threadIdx.x == 0) {
    its = items[blockIdx.x];
    Ds = insts[its.inst];
  }
  __syncthreads();
  const B32Item& it = its;  // descriptors in shared memory, read where used
  const B32Inst& D = Ds;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int M0 = D.M[0], M1 = D.M[1], n0 = D.n[0], n1 = D.n[1];
  const int ns0 = n0 - P, ns1 = n1 - (D.dim >= 2 ? P : 0);
  float* vb = sm;
  int* sx = reinterpret_cast<int*>(vb + r4(cap.vb));
  int* sy = sx + r4(cap.sx);
  float* vy = reinterpret_cast<float*>(sy + r4(cap.sy));
  int* ysp = reinterpret_cast<int*>(vy + r4(cap.vy));
  float* f = reinterpret_cast<float*>(ysp + r4(cap.ysp)) + (size_t)w * b32_warp_floats(cap, MODE);
  B32Warp L{};
  L.stage = f;
  f += 2 * r4(cap.stage);
  if (MODE != B32_RESIDUAL) {
    L.xr = f;
    f += r4(cap.xr);
    L.ring = f;
    f += r4(cap.ring);
  }
  if (MODE != B32_PROJECT) {
    L.dzy = f;
  }
  {
    const float* v0 = D.vals[0] + (long long)D.kbase[0] * (P + 1);
    for (int i = threadIdx.x; i < M0 * (P + 1); i += blockDim.x) {
      const int k = i / (P + 1), c = i - k * (P + 1);
      vb[k * W + c] = __ldg(v0 + i);
    }
    for (int j = threadIdx.x; j <= ns0; j += blockDim.x)
      sx[j] = j == ns0 ? M0 : __ldg(D.sstart[0] + D.cbase[0] + j) - D.kbase[0];
    if (D.dim >= 2) {
      const float* v1 = D.vals[1] + (long long)D.kbase[1] * (P + 1);
      for (int i = threadIdx.x; i < M1 * (P + 1); i += blockDim.x) {
        const int k = i / (P + 1), c = i - k * (P + 1);
        vy[k * W + c] = __ldg(v1 + i);
      }
      for (int k = threadIdx.x; k < M1; k += blockDim.x) ysp[k] = __ldg(D.span[1] + D.kbase[1] + k) - D.cbase[1];
      for (int j = threadIdx.x; j <= ns1; j += blockDim.x)
        sy[j] = j == ns1 ? M1 : __ldg(D.sstart[1] + D.cbase[1] + j) - D.kbase[1];
    } else if (threadIdx.x < W) {
      vy[threadIdx.x] = threadIdx.x == 0 ? 1.f : 0.f;  // 1-D: one row of weight 1
      if (threadIdx.x == 0) ysp[0] = 0;
    }
  }
  __syncthreads();
  const B32Tables T{vb, sx, sy, vy, ysp};
  int ra = 0, rb = 0, sa = 0, sb = ns1;
  if (w < it.nw) {
    if (D.dim == 3) {
      const int planes = (it.r1 - it.r0) / M1;
      ra = it.r0 + (planes * w / it.nw) * M1;
      rb = it.r0 + (planes * (w + 1) / it.nw) * M1;
    } else if (D.dim == 2) {
      sa = ns1 * w / it.nw;
      sb = ns1 * (w + 1) / it.nw;
      ra = sy[sa];
      rb = sy[sb];
    } else {
      rb = 1;
    }
  }
  float s2 = 0.f, emax = 0.f;
  if (ra < rb) b32_warp<P, MODE>(D, it, L, T, w, ra, rb, sa, sb, cap.stage, Q, P32, DZ, X, R, Z, s2, emax);
  if (MODE == B32_RESIDUAL) {
    double a = s2, b = emax;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
      red[w][0] = a;
      red[w][1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ta = 0.0, tb = 0.0;
      for (int k = 0; k < kB32Threads / 32; ++k) {
        ta += red[k][0];
        tb = fmax(tb, red[k][1]);
      }
      part[2 * ((long long)base + blockIdx.x)] = ta;
      part[2 * ((long long)base + blockIdx.x) + 1] = tb;
    }
  } else if (D.dim == 2 && it.nw > 1) {
    // y control points at the warps' boundaries: the earlier warp's part plus the later one's
    __syncthreads();
    const int per = P * n0;
    for (int t = threadIdx.x; t < (it.nw - 1) * per; t += blockDim.x) {
      const int wr = t / per + 1, rem = t - (wr - 1) * per;
      const int c = rem / n0, j0 = rem - c * n0;
      const int sw = ns1 * wr / it.nw;
      const float v = Z[it.z_off + ((long long)(2 * (wr - 1) + 1) * P + c) * n0 + j0] +
                      Z[it.z_off + ((long long)(2 * wr) * P + c) * n0 + j0];
      X[D.x_off + (long long)(sw + c) * n0 + j0] = ff(v);
    }
  }
}

template <int MODE>
void launch_mode(const B32Inst* insts, const B32Item* items, const int* first, const B32Caps* caps, const float* Q,
                 const float* P32, const float* DZ, ff* X, float* R, float* Z, double* part, cudaStream_t st,
                 const cudaStream_t* sides, int nsides, int& k, int only) {
#define MFA_B32_LAUNCH(PP)                                                                            \
  if ((only == 0 || only == PP) && first[PP] > first[PP - 1]) {                                      \
    const size_t smem = b32_smem_bytes(caps[PP], MODE);                                              \
    ensure_smem(k_b32<PP, MODE>, smem);                                                              \
    cudaStream_t s_ = nsides > 0 ? sides[k++ % nsides] : st;                                         \
    k_b32<PP, MODE><<<first[PP] - first[PP - 1], kB32Threads, smem, s_>>>(                           \
        insts, items + first[PP - 1], first[PP - 1], caps[PP], Q, P32, DZ, X, R, Z, part);           \
  }
  MFA_B32_LAUNCH(1) MFA_B32_LAUNCH(2) MFA_B32_LAUNCH(3) MFA_B32_LAUNCH(4) MFA_B32_LAUNCH(5) MFA_B32_LAUNCH(6)
  MFA_B32_LAUNCH(7)
#undef MFA_B32_LAUNCH
}

}  // namespace

size_t b32_smem_bytes(const B32Caps& cap, int mode) {
  return sizeof(float) * ((size_t)b32_cta_floats(cap) + (size_t)(kB32Threads / 32) * b32_warp_floats(cap, mode));
}

void launch_b32(int mode, const B32Inst* insts, const B32Item* items, const int* first, const B32Caps* caps,
                const float* Q, const float* P32, const float* DZ, ff* X, float* R, float* Z, double* part,
                cudaStream_t st, const cudaStream_t* sides, int nsides, int* next_side, int only_degree) {
  int k0 = next_side ? *next_side : 0;
  int& k = next_side ? *next_side : k0;
  if (mode == B32_PROJECT)
    launch_mode<B32_PROJECT>(insts, items, first, caps, Q, nullptr, nullptr, X, R, Z, nullptr, st, sides, nsides, k,
                             only_degree);
  else if (mode == B32_REFINE)
    launch_mode<B32_REFINE>(insts, items, first, caps, Q, P32, DZ, X, R, Z, nullptr, st, sides, nsides, k,
                            only_degree);
  else
    launch_mode<B32_RESIDUAL>(insts, items, first, caps, Q, P32, DZ, nullptr, nullptr, nullptr, part, st, sides,
                              nsides, k, only_degree);
}

// Over tiles of control points (first value, count): P32 = float(X), after
// X += dX where dX is given (the refinement's correction).  The same
// operations as k_b32_add followed by the whole-buffer cast.
__global__ void k_b32_cast_tiles(const long long* __restrict__ off, const int* __restrict__ len,
                                 ff* __restrict__ X, const ff* __restrict__ dX, float* __restrict__ P32) {
  const long long o = off[blockIdx.x];
  const int n = len[blockIdx.x];
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    ff x = X[o + t];
    if (dX) {
      x = x + dX[o + t];
      X[o + t] = x;
    }
    P32[o + t] = (float)x;
  }
}

void launch_b32_cast_tiles(const long long* off, const int* len, int ntiles, ff* X, const ff* dX, float* P32,
                           cudaStream_t st) {
  if (ntiles <= 0) return;
  k_b32_cast_tiles<<<ntiles, 256, 0, st>>>(off, len, X, dX, P32);
}

// z expansion of the FP32 control points of 3-D instances for the decode of
// the refinement and the residual: DZ[k2][j1][j0] = sum over c of
// N_{s+c}(u_{k2}) P32[s + c][j1][j0], s the z span of point k2 (FP32 in c
// order, as the decode's own expansion would take it), in the layout of R.
__global__ void __launch_bounds__(256) k_b32_zexpand(const B32Inst* __restrict__ insts,
                                                     const int* __restrict__ tile_inst,
                                                     const long long* __restrict__ tile_base,
                                                     const float* __restrict__ P32, float* __restrict__ DZ) {
  const B32Inst& D = insts[tile_inst[blockIdx.x]];
  const long long plane_cp = (long long)D.n[1] * D.n[0];
  const long long total = (long long)D.M[2] * plane_cp;
  const long long e = tile_base[blockIdx.x] + threadIdx.x;
  if (e >= total) return;
  const long long k2 =
      total <= 0xffffffffLL ? (long long)((unsigned)e / (unsigned)plane_cp) : e / plane_cp;
  const long long gk = D.kbase[2] + k2;
  const int sz = __ldg(D.span[2] + gk) - D.cbase[2];
  const float* src = P32 + D.x_off + sz * plane_cp + (e - k2 * plane_cp);
  const float* vz = D.vals[2] + gk * (D.p + 1);
  constexpr int PM = MFA_MAX_DEGREE;
  float g[PM + 1];  // every load in flight before the first product
#pragma unroll
  for (int c = 0; c <= PM; ++c) g[c] = c <= D.p ? __ldg(src + c * plane_cp) : 0.f;
  float a = 0.f;
#pragma unroll
  for (int c = 0; c <= PM; ++c)
    if (c <= D.p) a = fmaf(__ldg(vz + c), g[c], a);
  DZ[D.r_off + e] = a;
}

void launch_b32_zexpand(const B32Inst* insts, const int* tile_inst, const long long* tile_base, int ntiles,
                        const float* P32, float* DZ, cudaStream_t st) {
  if (ntiles <= 0) return;
  k_b32_zexpand<<<ntiles, 256, 0, st>>>(insts, tile_inst, tile_base, P32, DZ);
}

// X += dX over n float-float values (the refinement's correction of the
// control points).
__global__ void k_b32_add(ff* __restrict__ X, const ff* __restrict__ dX, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    X[i] = X[i] + dX[i];
}

void launch_b32_add(ff* X, const ff* dX, long long n, cudaStream_t st) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  const long long capb = 8LL * device_sm_count();
  if (blocks > capb) blocks = capb;
  k_b32_add<<<(unsigned)blocks, 256, 0, st>>>(X, dX, n);
}

// z contraction of the xy-reduced planes of 3-D instances: one thread per
// (j1, j0) column walks the planes k2 in order with the p + 1 z control
// points that plane touches open in registers, and writes each one (as
// float-float) once no later plane touches it, so every plane value is read
// once.  Control point (j0, j1, j2) = sum over planes k2 of
// N_{j2}(u_{k2}) R[k2][j1][j0] (FP32, planes in order).
__global__ void __launch_bounds__(kB32ZThreads) k_b32_zcontract(const B32Inst* __restrict__ insts,
                                                                const int* __restrict__ tile_inst,
                                                                const long long* __restrict__ tile_base,
                                                                const float* __restrict__ R, ff* __restrict__ X) {
  constexpr int PM = MFA_MAX_DEGREE;
  const B32Inst& D = insts[tile_inst[blockIdx.x]];
  const long long plane = (long long)D.n[0] * D.n[1];
  const long long col = tile_base[blockIdx.x] + threadIdx.x;
  if (col >= plane) return;
  const int p = D.p, n2 = D.n[2], M2 = D.M[2];
  const int* sp = D.span[2] + D.kbase[2];
  const float* vz = D.vals[2] + (long long)D.kbase[2] * (p + 1);
  const float* Rp = R + D.r_off + col;
  ff* Xp = X + D.x_off + col;
  float a[PM + 1];
#pragma unroll
  for (int c = 0; c <= PM; ++c) a[c] = 0.f;
  int cc = 0;  // first open z control point
  // planes in groups of kZGroup, the group's values loaded before its first
  // use (one column's planes are a stride apart: each load waits on DRAM)
  constexpr int kZGroup = 8;
  for (int k0 = 0; k0 < M2; k0 += kZGroup) {
    float rq[kZGroup];
#pragma unroll
    for (int u = 0; u < kZGroup; ++u) rq[u] = k0 + u < M2 ? __ldg(Rp + (long long)(k0 + u) * plane) : 0.f;
#pragma unroll
    for (int u = 0; u < kZGroup; ++u) {
      const int k = k0 + u;
      if (k >= M2) break;
      const int sk = __ldg(sp + k) - D.cbase[2];
      while (cc < sk) {
        Xp[(long long)cc * plane] = ff(a[0]);
#pragma unroll
        for (int c = 0; c < PM; ++c) a[c] = a[c + 1];
        a[PM] = 0.f;
        ++cc;
      }
      const float* v = vz + (long long)k * (p + 1);
#pragma unroll
      for (int c = 0; c <= PM; ++c)
        if (c <= p) a[c] = fmaf(__ldg(v + c), rq[u], a[c]);
    }
  }
#pragma unroll
  for (int c = 0; c <= PM; ++c)
    if (c <= p && cc + c < n2) Xp[(long long)(cc + c) * plane] = ff(a[c]);
  for (int j = cc + p + 1; j < n2; ++j) Xp[(long long)j * plane] = ff(0.f);  // spans without planes
}

void launch_b32_zcontract(const B32Inst* insts, const int* tile_inst, const long long* tile_base, int ntiles,
                          const float* R, ff* X, cudaStream_t st) {
  if (ntiles <= 0) return;
  k_b32_zcontract<<<ntiles, kB32ZThreads, 0, st>>>(insts, tile_inst, tile_base, R, X);
}

// Per instance, its items' totals in item order: out[2 i] = sum E^2,
// out[2 i + 1] = max |E| (the totals of instance i are parts range[2 i] ..
// range[2 i + 1] - 1).
__global__ void k_b32_reduce(const int* __restrict__ range, int count, const double* __restrict__ part,
                             double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double s = 0.0, m = 0.0;
  for (int k = range[2 * i]; k < range[2 * i + 1]; ++k) {
    s += part[2 * (long long)k];
    m = fmax(m, part[2 * (long long)k + 1]);
  }
  out[2 * i] = s;
  out[2 * i + 1] = m;
}

void launch_b32_reduce(const int* range, int count, const double* part, double* out, cudaStream_t st) {
  if (count <= 0) return;
  k_b32_reduce<<<(count + 127) / 128, 128, 0, st>>>(range, count, part, out);
}

}  // namespace mfa
