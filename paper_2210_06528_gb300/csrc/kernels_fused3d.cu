// Fused 3-D kernels for the data passes of the encode (Algorithm 1 setup and
// error steps), specialised on the degree P.
//
// Accumulation: `AccFF` keeps float-float sums (products formed exactly with
// FMA, sums compensated).  The kernels read the data once per subdomain window
// and stream it through shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>

#include "mfa_internal.cuh"

namespace mfa {

// ---------------------------------------------------------------------------
// accumulation policies
// ---------------------------------------------------------------------------

struct AccFF {
  using V = ff;
  __device__ static V zero() { return ff(0.f, 0.f); }
  // acc += (nh + nl) * x, low word unnormalised until finish()
  __device__ __forceinline__ static void add_v(V& acc, float nh, float nl, V x) { ff_acc_prod(acc, nh, nl, x); }
  __device__ __forceinline__ static V finish(V a) { return ff_norm(a); }
};


// ---------------------------------------------------------------------------
// Projection B_L = (N_z^T x N_y^T x N_x^T) Q over every window (the N^T Q
// assembly of the local normal equations, Eq. minimization-problem).
//
// One CTA per subdomain streams its window in batches of ZB z-planes.  A batch
// is one box of the data [ZB][BY][BX] copied by the tensor memory accelerator
// (or, for unaligned or FP64 input, by per-element asynchronous copies into
// the same layout): the box starts at the window's first x rounded down to a
// multiple of four, so point k of a row sits at staged position cx + k, and
// the positions outside the window carry zero basis values.  Rows are BX
// floats apart with BX = 4 (mod 8), so a warp's 16-byte row reads are free of
// bank conflicts.
//   stage 1 (x): one thread per data row; a sliding window of P+1
//                accumulators walks the row four points at a time, each point
//                adding its P+1 basis products; a control point is emitted
//                (in place, over consumed data) when the span moves past it.
//   stage 2 (y): one thread per output (plane, y-control point, x-control
//                point), summing the rows of the P+1 spans that support it.
//   stage 3 (z): every thread owns NPAIR (x,y) control-point pairs and keeps
//                a ring of P+1 accumulators per pair across the planes; a
//                z-control point is written to B_L when the planes' span
//                moves past it.
// Every product is (basis hi + lo) x value with an exact FMA product and a
// compensated (TwoSum) accumulation.
// ---------------------------------------------------------------------------

constexpr int kProjMaxSplit = 8;  // units per window along z, at most
constexpr int kS2C = 8;           // projection stage 2: x-control points per lane (even)

// First plane of unit b of a window of m2 planes cut into K units of whole
// batches of zb planes (unit K ends at m2).
__host__ __device__ inline int proj_unit_start(int m2, int zb, int K, int b) {
  const int nbat = (m2 + zb - 1) / zb;
  const int z = zb * ((b * nbat) / K);
  return b >= K || z > m2 ? m2 : z;
}

struct Proj3dArgs {
  LayoutDev L;
  const long long* offL;
  int zb;        // planes per batch (box z)
  int lx_shift;  // stage 2: log2 of the lanes per (plane, y-control point) group, 2^shift >= max L along x
  int bx;        // staged row pitch in floats = box x; multiple of 4, = 4 (mod 8)
  int by;        // staged rows per plane = box y = largest window along y
  int mz;        // largest window along z
  int n0, n1;    // largest L along x and y
  const AxisOp* inst;  // independent fits: the projection operand of every instance (data offset, strides)
  const int* order;    // CTA -> subdomain / instance (largest first), or null
  int ksplit;          // units per window along z (CTA b: subdomain b % nsub, unit b / nsub)
  ff* zpart;           // partial sums of the z-control points two units share (ksplit > 1)
  unsigned* zctr;      // units finished per subdomain (zeroed before the launch)
  int pstride;         // stride of a z-control point's (x, y) pairs in zpart
  const int2* units;   // when set, CTA b takes unit units[b] = (subdomain, unit along z)
};

// Shared-memory carve-up of the projection, used by the kernel and the launcher.
// The basis lanes are padded to an even count WP so they pair up.
struct ProjSmem {
  size_t t2h, t2l, txh, txn, txl, ty, tz, spx, spy, spz, bar, total;
  int npp;  // stride of a plane of the stage-2 output (even)
};
__host__ __device__ inline ProjSmem proj_smem_layout(int W, int zb, int bx, int by, int mz, int n0, int n1) {
  ProjSmem s;
  auto al = [](size_t o) { return (o + 15) & ~size_t(15); };
  const int WP = 2 * ((W + 1) / 2);
  s.npp = (n0 * n1 + 1) & ~1;
  size_t o = (size_t)zb * by * bx * 4;  // staged data at offset 0 (128-byte aligned base)
  s.t2h = al(o);
  s.t2l = s.t2h + (size_t)zb * s.npp * 4;
  s.txh = al(s.t2l + (size_t)zb * s.npp * 4);
  s.txn = al(s.txh + (size_t)bx * WP * 4);
  s.txl = al(s.txn + (size_t)bx * WP * 4);
  s.ty = al(s.txl + (size_t)bx * WP * 4);
  s.tz = s.ty + (size_t)by * W * 16;
  s.spx = s.tz + (size_t)mz * W * 16;
  s.spy = s.spx + (size_t)bx * 4;
  s.spz = s.spy + (size_t)by * 4;
  s.bar = al(s.spz + (size_t)mz * 4);
  s.total = s.bar + 16;
  return s;
}

// NPR pairs of basis lanes of one table row (16-byte aligned when NPR = 2)
template <int NPR>
__device__ __forceinline__ void load_pairs(const float* t, float2* v) {
  if constexpr (NPR == 2) {
    const float4 a = *reinterpret_cast<const float4*>(t);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
  } else {
#pragma unroll
    for (int k = 0; k < NPR; ++k) v[k] = reinterpret_cast<const float2*>(t)[k];
  }
}

// Lane r of a window of W float-float accumulators held as pairs.
template <int R>
__device__ __forceinline__ ff ff2_lane(const ff2* w) {
  if constexpr (R & 1)
    return ff(w[R >> 1].hi.y, w[R >> 1].lo.y);
  else
    return ff(w[R >> 1].hi.x, w[R >> 1].lo.x);
}

// Slide a window of W paired accumulators by one: lane r takes lane r + 1,
// lane W - 1 (and the padding lane of an odd W) restarts at zero.
template <int W>
__device__ __forceinline__ void ff2_shift(ff2* w) {
  constexpr int NPR = (W + 1) / 2;
#pragma unroll
  for (int k = 0; k < NPR; ++k) {
    w[k].hi.x = w[k].hi.y;
    w[k].lo.x = w[k].lo.y;
    if (k + 1 < NPR) {
      w[k].hi.y = w[k + 1].hi.x;
      w[k].lo.y = w[k + 1].lo.x;
    } else {
      w[k].hi.y = 0.f;
      w[k].lo.y = 0.f;
    }
  }
  if constexpr (W & 1) {
    w[NPR - 1].hi.x = 0.f;
    w[NPR - 1].lo.x = 0.f;
  }
}

// Stage-1 output of x-control point c in a staged row: control points pair up
// in 16-byte groups (hi of 2k, hi of 2k+1, lo of 2k, lo of 2k+1), so stage 2
// reads two control points' values as ready-made lane pairs.
__device__ __forceinline__ void emit_x_cp(float* row, int c, ff v) {
  const ff f = fast_two_sum(v.hi, v.lo);
  float* b = row + 4 * (c >> 1) + (c & 1);
  b[0] = f.hi;
  b[2] = f.lo;
}

__device__ __forceinline__ void cp_async_f32(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Arm the barrier for `bytes` and start the copy of one [z][y][x] box at
// global coordinates (x, y, z) into `dst`.
__device__ __forceinline__ void tma_load_box(const CUtensorMap* map, float* dst, unsigned long long* bar, int x,
                                             int y, int z, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Wait for phase `parity` of the barrier; gives up after about two seconds of
// clock cycles and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 4000000000LL) return false;
  }
}

// Per-element staging of planes z0 .. z0+nz-1 (rows y < m1) into the box
// layout, for input the tensor copy cannot take: staged position i of a row
// holds global x = xa + i, zero beyond the grid.
template <typename TQ>
__device__ __forceinline__ void stage_rows(float* Qs, const TQ* Q, long long M0, long long M01, int xa, int y0,
                                           int z0, int nz, int m1, int bx, int by) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int row = warp; row < nz * m1; row += nwarp) {
    const int zz = row / m1, y = row - zz * m1;
    const TQ* src = Q + M01 * (z0 + zz) + M0 * (y0 + y);
    float* dst = Qs + (size_t)(zz * by + y) * bx;
    for (int i = lane; i < bx; i += 32) {
      const long long g = xa + i;
      if (g >= M0)
        dst[i] = 0.f;
      else if constexpr (sizeof(TQ) == 4)
        cp_async_f32(dst + i, reinterpret_cast<const float*>(src) + g);
      else
        dst[i] = (float)src[g];
    }
  }
  cp_async_commit();
}

template <int P, int NT, int NPAIR, bool TMA, typename TQ>
__global__ void __launch_bounds__(NT, 2) k_project3d_ff(const __grid_constant__ CUtensorMap tmq, Proj3dArgs A,
                                                         const TQ* __restrict__ Q, ff* __restrict__ BL,
                                                         int* status) {
  constexpr int W = P + 1;
  constexpr int NPR = (W + 1) / 2, WP = 2 * NPR;  // basis lanes in pairs
  constexpr int NS = NPAIR / 2;                    // stage-3 slots of two adjacent (x, y) pairs
  static_assert(NPAIR % 2 == 0, "pairs come in twos");
  extern __shared__ __align__(128) unsigned char smem[];
  const LayoutDev& L = A.L;
  const int K = A.ksplit;
  int s, kunit;
  if (A.units) {
    const int2 u = A.units[blockIdx.x];
    s = u.x;
    kunit = u.y;
  } else {
    s = A.order ? A.order[blockIdx.x] : (int)(blockIdx.x % (unsigned)L.nsub);
    kunit = A.order ? 0 : (int)(blockIdx.x / (unsigned)L.nsub);
  }
  int s0, s1, s2;
  sub_pieces(L, s, s0, s1, s2);
  const AxisSub bx = L.ax[0].subs[s0], by = L.ax[1].subs[s1], bz = L.ax[2].subs[s2];
  const int m0 = bx.m, m1 = by.m, m2 = bz.m;
  const int n0 = bx.nL, n1 = by.nL, n2 = bz.nL;
  const int zb = A.zb, BX = A.bx, BY = A.by;
  // the window's planes split into K units of whole batches (the host checks
  // that every unit keeps more than P+1 knot spans); this CTA takes unit
  // kunit, planes [zbnd[k], zbnd[k+1])
  __shared__ int zbnd[kProjMaxSplit + 1];
  __shared__ int last_unit;
  if (threadIdx.x < K + 1) zbnd[threadIdx.x] = proj_unit_start(m2, zb, K, threadIdx.x);
  // window origin in the data: the subdomain's corner of the one grid, or
  // (independent fits) the instance's own grid at its offset and strides
  long long M0 = L.M[0], M01 = L.M[0] * L.M[1];
  int wx = bx.k0, wy = by.k0, wz = bz.k0;
  if (A.inst) {
    const View& v = A.inst[s].in;
    Q += v.off;
    M0 = v.st[1];
    M01 = v.st[2];
    wx = wy = wz = 0;
  }
  const int cx = TMA ? (wx & 3) : 0;     // staged position of window point 0
  const int xa = wx - cx;                // data x of staged position 0 (multiple of 4 for the tensor copy)
  const int nq4 = (cx + m0 + 3) >> 2;    // 16-byte chunks of a row that hold window points
  const ProjSmem lay = proj_smem_layout(W, zb, BX, BY, A.mz, A.n0, A.n1);
  const int npp = lay.npp;

  float* Qs = reinterpret_cast<float*>(smem);  // [zb][BY][BX]; row t's stage-1 output in 16-byte groups at its start
  float* T2h = reinterpret_cast<float*>(smem + lay.t2h);  // [zb][npp] hi words of the stage-2 output
  float* T2l = reinterpret_cast<float*>(smem + lay.t2l);  // lo words
  float* txh = reinterpret_cast<float*>(smem + lay.txh);  // [BX][WP] x basis by staged position: hi
  float* txn = reinterpret_cast<float*>(smem + lay.txn);  //   -hi
  float* txl = reinterpret_cast<float*>(smem + lay.txl);  //   lo
  float4* ty = reinterpret_cast<float4*>(smem + lay.ty);  // [m1][W] {hi, -hi, lo, 0}
  float4* tz = reinterpret_cast<float4*>(smem + lay.tz);  // [m2][W]
  int* spx = reinterpret_cast<int*>(smem + lay.spx);      // [BX] local span by staged position
  int* spy = reinterpret_cast<int*>(smem + lay.spy);
  int* spz = reinterpret_cast<int*>(smem + lay.spz);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + lay.bar);
  const unsigned box_bytes = (unsigned)(zb * BY * BX * 4);

  __syncthreads();  // unit bounds
  const int za = zbnd[kunit], zend = zbnd[kunit + 1];
  if constexpr (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      tma_load_box(&tmq, Qs, bar, xa, wy, wz + za, box_bytes);
    }
  } else {
    stage_rows<TQ>(Qs, Q, M0, M01, xa, wy, wz + za, min(zb, zend - za), m1, BX, BY);
  }

  // basis tables: x by staged position (zero outside the window and in the
  // padding lane, span held at the nearest window point so no control point
  // is emitted there)
  const ff* vx = L.ax[0].vals_ff;
  const ff* vy = L.ax[1].vals_ff;
  const ff* vz = L.ax[2].vals_ff;
  for (int i = threadIdx.x; i < BX; i += NT) {
    const int k = i - cx;
    const bool in = k >= 0 && k < m0;
    const int kk = min(max(k, 0), m0 - 1);
    spx[i] = L.ax[0].span[bx.k0 + kk] - bx.l0;
#pragma unroll
    for (int r = 0; r < WP; ++r) {
      const ff v = in && r < W ? vx[(long long)(bx.k0 + k) * W + r] : ff(0.f, 0.f);
      txh[i * WP + r] = v.hi;
      txn[i * WP + r] = -v.hi;
      txl[i * WP + r] = v.lo;
    }
  }
  for (int i = threadIdx.x; i < m1; i += NT) {
    const int k = by.k0 + i;
    spy[i] = L.ax[1].span[k] - by.l0;
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const ff v = vy[(long long)k * W + r];
      ty[i * W + r] = make_float4(v.hi, -v.hi, v.lo, 0.f);
    }
  }
  for (int i = threadIdx.x; i < m2; i += NT) {
    const int k = bz.k0 + i;
    spz[i] = L.ax[2].span[k] - bz.l0;
#pragma unroll
    for (int r = 0; r < W; ++r) {
      const ff v = vz[(long long)k * W + r];
      tz[i * W + r] = make_float4(v.hi, -v.hi, v.lo, 0.f);
    }
  }

  // stage-3 ring: slot j holds the (x, y) pairs q0 = 2 (threadIdx.x + j NT)
  // (lane x) and q0 + 1 (lane y), entry r the z-control point curz + r
  ff2 ring[NS][W];
#pragma unroll
  for (int j = 0; j < NS; ++j)
#pragma unroll
    for (int r = 0; r < W; ++r) ring[j][r] = ff2_zero();
  const int npairs = n0 * n1;
  ff* out = BL + A.offL[s];
  bool bad = false;
  unsigned phase = 0;
  __syncthreads();     // tables written, barrier initialised
  int curz = spz[za];  // z-control point held in ring entry 0
  // z-control points this unit shares with the previous unit ([hlo, hhi],
  // at most P+1 of them) and with the next ([tlo, ...]): their sums go to
  // partial slots
  const int hlo = spz[za], hhi = kunit > 0 ? spz[za - 1] + P : hlo - 1;
  const int tlo = kunit < K - 1 ? spz[zend] : INT_MAX;
  const int pst = A.pstride;
  auto zdst = [&](int c, int q) -> ff* {
    if (c <= hhi) return A.zpart + ((size_t)(s * (K - 1) + kunit - 1) * 2 + 1) * W * pst + (size_t)(c - hlo) * pst + q;
    if (c >= tlo) return A.zpart + ((size_t)(s * (K - 1) + kunit) * 2 + 0) * W * pst + (size_t)(c - tlo) * pst + q;
    return out + (long long)c * npairs + q;
  };

  for (int z0 = za; z0 < zend; z0 += zb) {
    const int nz = min(zb, zend - z0);
    bool lost = false;
    if constexpr (TMA) {
      lost = !mbar_wait(bar, phase);
      phase ^= 1u;
    } else {
      cp_async_wait_all();
    }
    if (__syncthreads_or(lost)) {
      if (threadIdx.x == 0) {
        if (status) atomicExch(status, MFA_ERR_TIMEOUT);
        if constexpr (TMA) mbar_wait(bar, phase ^ 1u);  // one more bounded wait for the copy in flight
      }
      return;
    }
    // ---- stage 1: one staged row per thread, four points per 16-byte read,
    // sliding window of P+1 accumulators in lane pairs; the output overwrites
    // the consumed part of the row
    for (int t = threadIdx.x; t < nz * m1; t += NT) {
      const int zz = t / m1, y = t - zz * m1;
      float* row = Qs + (size_t)(zz * BY + y) * BX;
      ff2 win[NPR];
#pragma unroll
      for (int k = 0; k < NPR; ++k) win[k] = ff2_zero();
      int cur = spx[0];
      for (int j = 0; j < nq4; ++j) {
        const float4 q4 = reinterpret_cast<const float4*>(row)[j];
        const int4 s4 = reinterpret_cast<const int4*>(spx)[j];  // spans of the chunk's four points
        const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
        const int sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * j + u;
          // the point's basis rows are read before a control point is emitted,
          // so their latency overlaps the emission
          float2 nh[NPR], nn[NPR], nl[NPR];
          load_pairs<NPR>(txh + i * WP, nh);
          load_pairs<NPR>(txn + i * WP, nn);
          load_pairs<NPR>(txl + i * WP, nl);
          // a point starts at most one new span (every span of a valid layout
          // holds a data point; the host checks it for the fused path)
          if (cur < sv[u]) {
            if (cur >= 0 && cur < n0) emit_x_cp(row, cur, ff2_lane<0>(win));
            ff2_shift<W>(win);
            ++cur;
          }
          const float2 x = dup2(qv[u]);
#pragma unroll
          for (int k = 0; k < NPR; ++k) ff2_add_f(win[k], nh[k], nn[k], nl[k], x);
        }
      }
      if (cur >= 0 && cur < n0) emit_x_cp(row, cur, ff2_lane<0>(win));
      if (cur + 1 >= 0 && cur + 1 < n0) emit_x_cp(row, cur + 1, ff2_lane<1>(win));
      if (cur + 2 >= 0 && cur + 2 < n0) emit_x_cp(row, cur + 2, ff2_lane<2>(win));
      if constexpr (W > 3)
        if (cur + 3 >= 0 && cur + 3 < n0) emit_x_cp(row, cur + 3, ff2_lane<3 % W>(win));
      if constexpr (W > 4)
        if (cur + 4 >= 0 && cur + 4 < n0) emit_x_cp(row, cur + 4, ff2_lane<4 % W>(win));
      if constexpr (W > 5)
        if (cur + 5 >= 0 && cur + 5 < n0) emit_x_cp(row, cur + 5, ff2_lane<5 % W>(win));
    }
    __syncthreads();
    // ---- stage 2 (gather form): one warp-aligned group of lanes per (plane,
    // y-control point), each lane S2C adjacent x-control points (S2C/2 lane
    // pairs, independent sums sharing each basis read); each output sums its
    // P+1 supporting spans' rows, so the work per output is even and no row is
    // read for a control point it does not touch
    {
      const int* ss = L.ax[1].span_start;
      const int sh = A.lx_shift;                 // lanes per group = 1 << sh >= n0 / S2C
      const int lmask = (1 << sh) - 1;
      const int lx = threadIdx.x & lmask;
      const int gstep = NT >> sh;                // groups advanced per pass
      int c1 = threadIdx.x >> sh, zz = 0;
      while (c1 >= n1) {
        c1 -= n1;
        ++zz;
      }
      for (; zz < nz; ) {
        if (kS2C * lx < n0) {
          const int g1 = by.l0 + c1;
          const int ys = max(ss[max(g1 - P, 0)] - by.k0, 0);
          const int ye = min(ss[min(g1, L.ax[1].nspans - 1) + 1] - by.k0, m1);
          const float* colf = Qs + (size_t)zz * BY * BX + 2 * kS2C * lx;
          ff2 a[kS2C / 2];
#pragma unroll
          for (int k = 0; k < kS2C / 2; ++k) a[k] = ff2_zero();
          for (int y = ys; y < ye; ++y) {
            const float4 nb = ty[y * W + (c1 - spy[y])];
            const float2 bh = dup2(nb.x), bn = dup2(nb.y), bl = dup2(nb.z);
#pragma unroll
            for (int k = 0; k < kS2C / 2; ++k) {
              const float4 u = *reinterpret_cast<const float4*>(colf + (size_t)y * BX + 4 * k);
              ff2_add_v(a[k], bh, bn, bl, make_float2(u.x, u.y), make_float2(u.z, u.w));
            }
          }
          const int o = zz * npp + c1 * n0 + kS2C * lx;
#pragma unroll
          for (int k = 0; k < kS2C / 2; ++k) {
            if (kS2C * lx + 2 * k < n0) {
              const ff r = AccFF::finish(ff(a[k].hi.x, a[k].lo.x));
              T2h[o + 2 * k] = r.hi;
              T2l[o + 2 * k] = r.lo;
            }
            if (kS2C * lx + 2 * k + 1 < n0) {
              const ff r = AccFF::finish(ff(a[k].hi.y, a[k].lo.y));
              T2h[o + 2 * k + 1] = r.hi;
              T2l[o + 2 * k + 1] = r.lo;
            }
          }
        }
        c1 += gstep;
        while (c1 >= n1) {
          c1 -= n1;
          ++zz;
        }
      }
    }
    // the staged rows are free again: order this CTA's shared-memory accesses
    // before the copy engine's writes, then fetch the next batch behind stage 3
    if constexpr (TMA) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (z0 + zb < zend) {
      if constexpr (TMA) {
        if (threadIdx.x == 0) tma_load_box(&tmq, Qs, bar, xa, wy, wz + z0 + zb, box_bytes);
      } else {
        stage_rows<TQ>(Qs, Q, M0, M01, xa, wy, wz + z0 + zb, min(zb, zend - z0 - zb), m1, BX, BY);
      }
    }
    // ---- stage 3: accumulate the planes into the z ring (the plane's basis
    // row and stage-2 values are read before a z-control point is emitted)
    for (int zz = 0; zz < nz; ++zz) {
      const int kz = z0 + zz;
      const int sz = spz[kz];
      float2 zh[W], zn[W], zl[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        const float4 b = tz[kz * W + r];
        zh[r] = dup2(b.x);
        zn[r] = dup2(b.y);
        zl[r] = dup2(b.z);
      }
      const float* th = T2h + zz * npp;
      const float* tl = T2l + zz * npp;
      float2 xh[NS], xl[NS];
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int q0 = min(2 * (threadIdx.x + j * NT), npp - 2);
        xh[j] = *reinterpret_cast<const float2*>(th + q0);
        xl[j] = *reinterpret_cast<const float2*>(tl + q0);
      }
      while (curz < sz) {
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          const int q0 = 2 * (threadIdx.x + j * NT);
          if (curz >= 0 && curz < n2) {
            if (q0 < npairs) {
              const ff v = AccFF::finish(ff(ring[j][0].hi.x, ring[j][0].lo.x));
              bad |= !isfinite(v.hi);
              *zdst(curz, q0) = v;
            }
            if (q0 + 1 < npairs) {
              const ff v = AccFF::finish(ff(ring[j][0].hi.y, ring[j][0].lo.y));
              bad |= !isfinite(v.hi);
              *zdst(curz, q0 + 1) = v;
            }
          }
#pragma unroll
          for (int r = 0; r < P; ++r) ring[j][r] = ring[j][r + 1];
          ring[j][P] = ff2_zero();
        }
        ++curz;
      }
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int q0 = 2 * (threadIdx.x + j * NT);
        if (q0 < npairs) {
#pragma unroll
          for (int r = 0; r < W; ++r) ff2_add_v(ring[j][r], zh[r], zn[r], zl[r], xh[j], xl[j]);
        }
      }
    }
    // T2 is rewritten by the next batch's stage 2 only after its stage-1 barrier
  }
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int q0 = 2 * (threadIdx.x + j * NT);
#pragma unroll
    for (int r = 0; r < W; ++r)
      if (curz + r >= 0 && curz + r < n2) {
        if (q0 < npairs) {
          const ff v = AccFF::finish(ff(ring[j][r].hi.x, ring[j][r].lo.x));
          bad |= !isfinite(v.hi);
          *zdst(curz + r, q0) = v;
        }
        if (q0 + 1 < npairs) {
          const ff v = AccFF::finish(ff(ring[j][r].hi.y, ring[j][r].lo.y));
          bad |= !isfinite(v.hi);
          *zdst(curz + r, q0 + 1) = v;
        }
      }
  }
  if (K > 1) {
    // the last unit of the subdomain to finish adds the partial sums of every
    // shared z-control point, the earlier planes' part first
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_unit = atomicAdd(&A.zctr[s], 1u) == (unsigned)(K - 1);
    __syncthreads();
    if (last_unit) {
      __threadfence();
      for (int b = 1; b < K; ++b) {
        const int zp = zbnd[b];
        const int lo = spz[zp], hi = min(spz[zp - 1] + P, n2 - 1);
        const ff* before = A.zpart + ((size_t)(s * (K - 1) + b - 1) * 2 + 0) * W * pst;
        const ff* after = before + (size_t)W * pst;
        for (int c = max(lo, 0); c <= hi; ++c)
          for (int q = threadIdx.x; q < npairs; q += NT) {
            const float2 u = __ldcg(reinterpret_cast<const float2*>(before + (size_t)(c - lo) * pst + q));
            const float2 w = __ldcg(reinterpret_cast<const float2*>(after + (size_t)(c - lo) * pst + q));
            const ff v = ff(u.x, u.y) + ff(w.x, w.y);
            bad |= !isfinite(v.hi);
            out[(long long)c * npairs + q] = v;
          }
      }
    }
  }
  if (bad && status) atomicExch(status, MFA_ERR_NONFINITE);
}

constexpr int kProjThreads = 256;

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Row pitch of the staged box: window plus alignment slack, room for the
// in-place output, a multiple of 4 floats with an odd number of 16-byte chunks.
static int proj_pitch(int maxm0, int maxn0) {
  // stage 2 reads the control points of a row in groups of kS2C (2 floats each)
  int bx = std::max(maxm0 + 3, 2 * kS2C * ((maxn0 + kS2C - 1) / kS2C));
  bx = (bx + 3) & ~3;
  if (bx % 8 == 0) bx += 4;
  return bx;
}

int proj3d_planes_per_batch(int P, int maxm0, int maxm1, int maxm2, int maxn0, int maxn1) {
  // fill the stage-1 rows onto the threads, then shrink until two CTAs fit an
  // SM (half its shared memory less the per-block reservation)
  static const size_t two_per_sm = [] {
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    return per_sm > 0 ? (size_t)(per_sm / 2 - reserved) : (size_t)110 * 1024;
  }();
  const int bx = proj_pitch(maxm0, maxn0);
  int zb = std::max(1, std::min(4, kProjThreads / std::max(maxm1, 1)));
  while (zb > 1 && proj_smem_layout(P + 1, zb, bx, maxm1, maxm2, maxn0, maxn1).total > two_per_sm) zb--;
  return zb;
}

int proj3d_unit_start(int m2, int zb, int K, int b) { return proj_unit_start(m2, zb, K, b); }

bool proj3d_split_ok(int P, int zb, int K, long long M, int nspans, long long k0, int m) {
  // every unit keeps more than P+1 knot spans, so no z-control point takes
  // planes of three units (span of point k: floor(k nspans / (M-1)), capped)
  auto span = [&](long long k) {
    const long long sk = M == 1 ? 0 : (k * nspans) / (M - 1);
    return sk > nspans - 1 ? (long long)nspans - 1 : sk;
  };
  for (int b = 0; b < K; ++b) {
    const int z0 = proj_unit_start(m, zb, K, b), z1 = proj_unit_start(m, zb, K, b + 1);
    if (z1 <= z0 || span(k0 + z1 - 1) - span(k0 + z0) + 1 < P + 2) return false;
  }
  return true;
}

// Returns false when the fused kernel does not cover this layout (the caller
// then runs the generic per-axis kernels).  `inplace_ok` says every x-window
// has at least two points per span, so the stage-1 output can overwrite the
// consumed data in place.
template <typename TQ>
bool launch_project3d_ff(const LayoutDev& L, const long long* offL, int maxm0, int maxm1, int maxm2, int maxn0,
                         int maxn1, bool inplace_ok, const TQ* Q, ff* BL, int* status, cudaStream_t st,
                         const AxisOp* inst, const int* order, int ksplit, ff* zpart, unsigned* zctr,
                         const int2* units, int nunits, bool first) {
  const int P = L.ax[0].p;
  if (L.dim != 3 || L.ax[1].p != P || L.ax[2].p != P || !inplace_ok) return false;
  const int npairs = maxn0 * maxn1;
  Proj3dArgs A;
  A.L = L;
  A.offL = offL;
  A.inst = inst;
  A.order = order;
  A.ksplit = (inst || order || !zpart || !zctr) ? 1 : std::max(1, std::min(ksplit, kProjMaxSplit));
  A.zpart = zpart;
  A.zctr = zctr;
  A.pstride = npairs;
  A.units = A.ksplit > 1 ? units : nullptr;
  if (A.units && nunits <= 0) return true;  // no unit in this part
  A.bx = proj_pitch(maxm0, maxn0);
  A.by = maxm1;
  A.mz = maxm2;
  A.n0 = maxn0;
  A.n1 = maxn1;
  A.zb = proj3d_planes_per_batch(P, maxm0, maxm1, maxm2, maxn0, maxn1);
  const int W = P + 1;
  const size_t smem = proj_smem_layout(W, A.zb, A.bx, A.by, A.mz, A.n0, A.n1).total;
  if (smem > 200 * 1024 || npairs > 8 * kProjThreads) return false;
  // stage 2: a group of 1 << lx_shift lanes covers the x-control points, kS2C per lane
  A.lx_shift = 0;
  while ((1 << A.lx_shift) < (maxn0 + kS2C - 1) / kS2C) ++A.lx_shift;
  if ((1 << A.lx_shift) > kProjThreads) return false;

  // the tensor copy takes FP32 data on a 16-byte aligned base with rows a
  // multiple of 16 bytes long and boxes of at most 256 per dimension
  CUtensorMap tmap;
  std::memset(&tmap, 0, sizeof(tmap));
  bool tma = !inst && sizeof(TQ) == 4 && (reinterpret_cast<uintptr_t>(Q) % 16) == 0 && L.M[0] % 4 == 0 &&
             A.bx <= 256 && A.by <= 256 && tensor_map_encoder() != nullptr;
  if (tma) {
    const cuuint64_t dims[3] = {(cuuint64_t)L.M[0], (cuuint64_t)L.M[1], (cuuint64_t)L.M[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)L.M[0] * 4, (cuuint64_t)(L.M[0] * L.M[1]) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)A.bx, (cuuint32_t)A.by, (cuuint32_t)A.zb};
    const cuuint32_t estr[3] = {1, 1, 1};
    tma = tensor_map_encoder()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<TQ*>(Q), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  auto go = [&](auto kernel) {
    ensure_smem(kernel, smem, true);
    if (A.ksplit > 1 && first) cudaMemsetAsync(zctr, 0, sizeof(unsigned) * L.nsub, st);
    kernel<<<A.units ? nunits : L.nsub * A.ksplit, kProjThreads, smem, st>>>(tmap, A, Q, BL, status);
  };
#define MFA_PROJ_NP(PP, NP)                                             \
  if constexpr (sizeof(TQ) == 4) {                                      \
    if (tma)                                                            \
      go(k_project3d_ff<PP, kProjThreads, NP, true, TQ>);               \
    else                                                                \
      go(k_project3d_ff<PP, kProjThreads, NP, false, TQ>);              \
  } else {                                                              \
    go(k_project3d_ff<PP, kProjThreads, NP, false, TQ>);                \
  }
#define MFA_PROJ_CASE(PP)                 \
  case PP:                                \
    if (npairs <= 4 * kProjThreads) {     \
      MFA_PROJ_NP(PP, 4)                  \
    } else {                              \
      MFA_PROJ_NP(PP, 8)                  \
    }                                     \
    return true;
  switch (P) {
    MFA_PROJ_CASE(2)
    MFA_PROJ_CASE(3)
    MFA_PROJ_CASE(4)
    MFA_PROJ_CASE(5)
    default:
      return false;
  }
#undef MFA_PROJ_CASE
#undef MFA_PROJ_NP
}

template bool launch_project3d_ff<float>(const LayoutDev&, const long long*, int, int, int, int, int, bool,
                                         const float*, ff*, int*, cudaStream_t, const AxisOp*, const int*, int, ff*,
                                         unsigned*, const int2*, int, bool);
template bool launch_project3d_ff<double>(const LayoutDev&, const long long*, int, int, int, int, int, bool,
                                          const double*, ff*, int*, cudaStream_t, const AxisOp*, const int*, int, ff*,
                                          unsigned*, const int2*, int, bool);

}  // namespace mfa

namespace mfa {

// ---------------------------------------------------------------------------
// Grid decode R P (Algorithm 1 error step) on tiles of TX x TY x TZ points,
// fused with either the residual E = Q - R P (per-CTA partial sums of E^2,
// max |E|, min Q, max Q) or a write of the decoded values.
//
// Per tile: load the (spans + P) control-point block, expand along z, then y,
// then x; every output sums P+1 float-float basis products.  The sums run on
// the paired FP32 instructions (ff2), two outputs per thread, with shared
// memory laid out so that each stage reads its lane pairs directly:
//   z: outputs at x-control points (2k, 2k+1); block hi and lo words apart;
//   y: outputs at rows y and y + TY/2 (gathered from the z stage);
//   x: the two rows of the y stage, stored as {hi y, hi y', lo y, lo y'}.
// ---------------------------------------------------------------------------

constexpr int kDecTX = 64, kDecTY = 8, kDecTZ = 8, kDecThreads = 256;
constexpr int kDecYH = kDecTY / 2;  // y rows pair as (y, y + kDecYH)
static_assert(kDecThreads / 32 == kDecTZ, "one warp per plane in the z expansion");
static_assert(kDecThreads == kDecTX * kDecYH, "x expansion: one thread per (x, row pair)");

// Shared-memory carve-up of the decode (floats): block hi/lo [ncz][ncy][ncxp],
// z stage hi/lo [TZ][ncy][ncxp], y stage float4 [TZ][TY/2][ncx], then the
// basis tables (hi, lo) and local spans of the tile's points.
struct DecSmem {
  size_t pbh, pbl, tzh, tzl, ty, tab, total;
};
__host__ __device__ inline DecSmem dec_smem_layout(int W, int ncx, int ncy, int ncz) {
  DecSmem d;
  const int ncxp = (ncx + 1) & ~1;
  const size_t blk = (size_t)ncz * ncy * ncxp * 4, tz = (size_t)kDecTZ * ncy * ncxp * 4;
  d.pbh = 0;
  d.pbl = d.pbh + blk;
  d.tzh = d.pbl + blk;
  d.tzl = d.tzh + tz;
  d.ty = (d.tzl + tz + 15) & ~size_t(15);
  d.tab = d.ty + (size_t)kDecTZ * kDecYH * ncx * 16;
  d.total = d.tab + (size_t)(2 * W + 1) * (kDecTX + kDecTY + kDecTZ) * 4;
  return d;
}

// floor(a / d) for 0 <= a < 1024 and 0 < d <= 128 by a multiply and a shift:
// with m = ceil(2^17 / d) the excess m d - 2^17 is below d <= 2^17 / 1024, so
// a m / 2^17 stays within 1/d above a / d and never crosses the next integer
// (integer only: no int/float conversions, which share the FP64 pipe)
__device__ __forceinline__ unsigned div_magic(unsigned d) { return ((1u << 17) + d - 1) / d; }
__device__ __forceinline__ int div_small(int a, unsigned m) { return (int)(((unsigned)a * m) >> 17); }

template <int P, typename V, typename TQ, typename TOut, bool RESID>
__global__ void __launch_bounds__(kDecThreads, (P >= 4 ? 3 : 4)) k_decode3d(LayoutDev L, const V* __restrict__ Pc,
                                                                            const TQ* __restrict__ Q,
                                                                            TOut* __restrict__ out,
                                                                            double* __restrict__ partials) {
  static_assert(sizeof(V) == sizeof(ff), "float-float control points");
  constexpr int W = P + 1;
  extern __shared__ __align__(128) unsigned char smem[];
  // one CTA per tile on a 3-D grid of tiles; the linear tile index names the
  // tile's residual partials
  const int tx = blockIdx.x, ty = blockIdx.y, tz = blockIdx.z;
  const int tile = tx + gridDim.x * (ty + gridDim.y * tz);
  const int x0 = tx * kDecTX, y0 = ty * kDecTY, z0 = tz * kDecTZ;
  const int x1 = min(x0 + kDecTX, (int)L.M[0]), y1 = min(y0 + kDecTY, (int)L.M[1]), z1 = min(z0 + kDecTZ, (int)L.M[2]);
  const int nx = x1 - x0, ny = y1 - y0, nz = z1 - z0;
  const AxisDev &ax = L.ax[0], &ay = L.ax[1], &az = L.ax[2];
  const int cx0 = ax.span[x0], cy0 = ay.span[y0], cz0 = az.span[z0];
  const int ncx = ax.span[x1 - 1] + W - cx0, ncy = ay.span[y1 - 1] + W - cy0, ncz = az.span[z1 - 1] + W - cz0;
  const int ncxp = (ncx + 1) & ~1;
  const DecSmem lay = dec_smem_layout(W, ncx, ncy, ncz);
  float* Pbh = reinterpret_cast<float*>(smem + lay.pbh);
  float* Pbl = reinterpret_cast<float*>(smem + lay.pbl);
  float* Tzh = reinterpret_cast<float*>(smem + lay.tzh);
  float* Tzl = reinterpret_cast<float*>(smem + lay.tzl);
  float4* Ty = reinterpret_cast<float4*>(smem + lay.ty);
  float* nxh = reinterpret_cast<float*>(smem + lay.tab);  // [TX][W]
  float* nxl = nxh + kDecTX * W;
  float* nyh = nxl + kDecTX * W;                          // [TY][W]
  float* nyl = nyh + kDecTY * W;
  float* nzh = nyl + kDecTY * W;                          // [TZ][W]
  float* nzl = nzh + kDecTZ * W;
  int* sx = reinterpret_cast<int*>(nzl + kDecTZ * W);     // local spans
  int* sy = sx + kDecTX;
  int* sz = sy + kDecTY;
  const ff* Pf = reinterpret_cast<const ff*>(Pc);

  if constexpr (RESID) {
    // bring the tile's data rows into L2 now; they are read after the z and
    // y expansions (one 128-byte line per thread: rows of up to 64 floats)
    constexpr int kLines = kDecTX * (int)sizeof(TQ) / 128;
    const int t = threadIdx.x;
    if (t < kDecTY * kDecTZ * kLines) {
      const int part = t % kLines, row = t / kLines;
      const int y = row % kDecTY, z = row / kDecTY;
      const int xs = part * (128 / (int)sizeof(TQ));
      if (y < ny && z < nz && xs < nx) {
        const TQ* a = Q + (long long)(x0 + xs) + L.M[0] * (y0 + y) + L.M[0] * L.M[1] * (z0 + z);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
      }
    }
  }
  // basis tables of the tile's points, zero (span 0) past the grid's end
  for (int i = threadIdx.x; i < kDecTX * W; i += kDecThreads) {
    const int k = i / W, r = i - k * W;
    const ff v = k < nx ? ax.vals_ff[(long long)(x0 + k) * W + r] : ff(0.f, 0.f);
    nxh[i] = v.hi;
    nxl[i] = v.lo;
    if (r == 0) sx[k] = k < nx ? ax.span[x0 + k] - cx0 : 0;
  }
  for (int i = threadIdx.x; i < kDecTY * W; i += kDecThreads) {
    const int k = i / W, r = i - k * W;
    const ff v = k < ny ? ay.vals_ff[(long long)(y0 + k) * W + r] : ff(0.f, 0.f);
    nyh[i] = v.hi;
    nyl[i] = v.lo;
    if (r == 0) sy[k] = k < ny ? ay.span[y0 + k] - cy0 : 0;
  }
  for (int i = threadIdx.x; i < kDecTZ * W; i += kDecThreads) {
    const int k = i / W, r = i - k * W;
    const ff v = k < nz ? az.vals_ff[(long long)(z0 + k) * W + r] : ff(0.f, 0.f);
    nzh[i] = v.hi;
    nzl[i] = v.lo;
    if (r == 0) sz[k] = k < nz ? az.span[z0 + k] - cz0 : 0;
  }
  // control-point block, hi and lo words apart: lanes along x, warps over
  // (z, y) rows of the block
  const long long n0 = L.ncp[0], n01 = L.ncp[0] * L.ncp[1];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;  // 8 groups of 32
  const bool small_rows = ncz * ncy < 1024 && ncy <= 128;  // div_small's range
  const unsigned rcy = div_magic(ncy);
  for (int row = grp; row < ncz * ncy; row += kDecThreads / 32) {
    const int cz = small_rows ? div_small(row, rcy) : row / ncy, cy = row - cz * ncy;
    const ff* src = Pf + (long long)cx0 + n0 * (cy0 + cy) + n01 * (cz0 + cz);
    for (int cx = lane; cx < ncxp; cx += 32) {
      const ff v = cx < ncx ? src[cx] : ff(0.f, 0.f);
      Pbh[row * ncxp + cx] = v.hi;
      Pbl[row * ncxp + cx] = v.lo;
    }
  }
  __syncthreads();
  // z expansion: warp w takes plane z = w; lanes over (y-control point,
  // x-control-point pair), two items in flight
  {
    const int z = grp;
    if (z < nz) {
      float2 bh[W], bn[W], bl[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        bh[r] = dup2(nzh[z * W + r]);
        bn[r] = dup2(-nzh[z * W + r]);
        bl[r] = dup2(nzl[z * W + r]);
      }
      const int szz = sz[z];
      const int npr = ncxp >> 1, nit = ncy * npr;
      const unsigned rcp = div_magic(npr);  // nit < 1024, npr <= 128 (tiles of at most 64 + P x-control points)
      const int pst = ncy * ncxp;  // plane stride of the block
      for (int it = lane; it < nit; it += 64) {
        const int it2 = min(it + 32, nit - 1);
        const int cya = div_small(it, rcp), ka = it - cya * npr;
        const int cyb = div_small(it2, rcp), kb = it2 - cyb * npr;
        const int oa = (szz * ncy + cya) * ncxp + 2 * ka, ob = (szz * ncy + cyb) * ncxp + 2 * kb;
        ff2 A = ff2_zero(), B = ff2_zero();
#pragma unroll
        for (int r = 0; r < W; ++r) {
          ff2_add_v(A, bh[r], bn[r], bl[r], *reinterpret_cast<const float2*>(Pbh + oa + r * pst),
                    *reinterpret_cast<const float2*>(Pbl + oa + r * pst));
          ff2_add_v(B, bh[r], bn[r], bl[r], *reinterpret_cast<const float2*>(Pbh + ob + r * pst),
                    *reinterpret_cast<const float2*>(Pbl + ob + r * pst));
        }
        {
          const ff a = fast_two_sum(A.hi.x, A.lo.x), b = fast_two_sum(A.hi.y, A.lo.y);
          const int to = (z * ncy + cya) * ncxp + 2 * ka;
          *reinterpret_cast<float2*>(Tzh + to) = make_float2(a.hi, b.hi);
          *reinterpret_cast<float2*>(Tzl + to) = make_float2(a.lo, b.lo);
        }
        if (it + 32 < nit) {
          const ff a = fast_two_sum(B.hi.x, B.lo.x), b = fast_two_sum(B.hi.y, B.lo.y);
          const int to = (z * ncy + cyb) * ncxp + 2 * kb;
          *reinterpret_cast<float2*>(Tzh + to) = make_float2(a.hi, b.hi);
          *reinterpret_cast<float2*>(Tzl + to) = make_float2(a.lo, b.lo);
        }
      }
    }
  }
  __syncthreads();
  // y expansion: rows yl and yl + TY/2 together; a thread keeps its yl and
  // has two (plane, x-control point) items in flight
  {
    constexpr int kPer = kDecThreads / kDecYH;  // threads per row pair
    const int yl = threadIdx.x / kPer, tl = threadIdx.x - yl * kPer;
    const int ya = yl, yb = yl + kDecYH;
    if (ya < ny) {
      float2 bh[W], bn[W], bl[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        bh[r] = make_float2(nyh[ya * W + r], nyh[yb * W + r]);
        bn[r] = make_float2(-nyh[ya * W + r], -nyh[yb * W + r]);
        bl[r] = make_float2(nyl[ya * W + r], nyl[yb * W + r]);
      }
      const int ra = sy[ya], rb = sy[yb];
      const int nit = nz * ncx;
      const unsigned rcp = div_magic(ncx);  // nit = nz * ncx < 1024, ncx <= 128
      for (int it = tl; it < nit; it += 2 * kPer) {
        const int it2 = min(it + kPer, nit - 1);
        const int za = div_small(it, rcp), ca = it - za * ncx;
        const int zb2 = div_small(it2, rcp), cb = it2 - zb2 * ncx;
        const float* ha = Tzh + za * ncy * ncxp + ca;
        const float* la = Tzl + za * ncy * ncxp + ca;
        const float* hb = Tzh + zb2 * ncy * ncxp + cb;
        const float* lb = Tzl + zb2 * ncy * ncxp + cb;
        ff2 A = ff2_zero(), B = ff2_zero();
#pragma unroll
        for (int r = 0; r < W; ++r) {
          ff2_add_v(A, bh[r], bn[r], bl[r], make_float2(ha[(ra + r) * ncxp], ha[(rb + r) * ncxp]),
                    make_float2(la[(ra + r) * ncxp], la[(rb + r) * ncxp]));
          ff2_add_v(B, bh[r], bn[r], bl[r], make_float2(hb[(ra + r) * ncxp], hb[(rb + r) * ncxp]),
                    make_float2(lb[(ra + r) * ncxp], lb[(rb + r) * ncxp]));
        }
        {
          const ff a = fast_two_sum(A.hi.x, A.lo.x), b = fast_two_sum(A.hi.y, A.lo.y);
          Ty[(za * kDecYH + yl) * ncx + ca] = make_float4(a.hi, b.hi, a.lo, b.lo);
        }
        if (it + kPer < nit) {
          const ff a = fast_two_sum(B.hi.x, B.lo.x), b = fast_two_sum(B.hi.y, B.lo.y);
          Ty[(zb2 * kDecYH + yl) * ncx + cb] = make_float4(a.hi, b.hi, a.lo, b.lo);
        }
      }
    }
  }
  __syncthreads();
  // x expansion of every point of the tile, then residual or output: thread
  // (xt, yl) evaluates rows yl and yl + TY/2, two planes at a time
  float s2 = 0.f, emax = 0.f, qmin = INFINITY, qmax = -INFINITY;
  const long long M0 = L.M[0], M01 = L.M[0] * L.M[1];
  const int xt = threadIdx.x & (kDecTX - 1), yt = threadIdx.x / kDecTX;
  // offset of this thread's point (x0 + xt, y0 + yt, z0 + z) in the grid:
  // a base at z = 0, plus a plane step per z and kDecYH rows for the second row
  const long long g0 = (long long)(x0 + xt) + M0 * (y0 + yt) + M01 * z0, gy = M0 * kDecYH;
  auto emit = [&](const ff2& acc, int z, long long gz) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int y = yt + hh * kDecYH;
      if (y >= ny) continue;
      const ff v = hh ? fast_two_sum(acc.hi.y, acc.lo.y) : fast_two_sum(acc.hi.x, acc.lo.x);
      const long long g = hh ? gz + gy : gz;
      if constexpr (RESID) {
        const float q = (float)Q[g];
        // E = q - (hi + lo): q - hi is exact when the fit is close (Sterbenz)
        const float e = __fsub_rn(__fsub_rn(q, v.hi), v.lo);
        s2 = fmaf(e, e, s2);
        emax = fmaxf(emax, fabsf(e));
        qmin = fminf(qmin, q);
        qmax = fmaxf(qmax, q);
      } else {
        // hi + lo is exact in FP64, so a float output is its FP32 rounding
        // (one FP32 add); a double output takes the exact sum
        if constexpr (sizeof(TOut) == 4)
          out[g] = __fadd_rn(v.hi, v.lo);
        else
          out[g] = (TOut)((double)v.hi + (double)v.lo);
      }
    }
  };
  if (xt < nx && yt < ny) {
    float2 bh[W], bn[W], bl[W];
#pragma unroll
    for (int r = 0; r < W; ++r) {
      bh[r] = dup2(nxh[xt * W + r]);
      bn[r] = dup2(-nxh[xt * W + r]);
      bl[r] = dup2(nxl[xt * W + r]);
    }
    const int sxx = sx[xt];
    long long gz = g0;  // offset at plane z
    for (int z = 0; z < nz; z += 2, gz += 2 * M01) {
      const int z2 = min(z + 1, nz - 1);
      const float4* sa = Ty + (z * kDecYH + yt) * ncx + sxx;
      const float4* sb = Ty + (z2 * kDecYH + yt) * ncx + sxx;
      ff2 A = ff2_zero(), B = ff2_zero();
#pragma unroll
      for (int r = 0; r < W; ++r) {
        const float4 ta = sa[r], tb = sb[r];
        ff2_add_v(A, bh[r], bn[r], bl[r], make_float2(ta.x, ta.y), make_float2(ta.z, ta.w));
        ff2_add_v(B, bh[r], bn[r], bl[r], make_float2(tb.x, tb.y), make_float2(tb.z, tb.w));
      }
      emit(A, z, gz);
      if (z + 1 < nz) emit(B, z + 1, gz + M01);
    }
  }
  if constexpr (RESID) {
    // block reduction into this tile's slot.  The extrema are exact in FP32
    // and the sum of squares moves as a float-float, so the whole reduction
    // runs on the FP32 pipes; only the four results are widened to FP64 (the
    // FP64 pipe of this GPU is a small fraction of the FP32 ones, and every
    // tile ends here)
    ff fs2(s2, 0.f);
    for (int o = 16; o > 0; o >>= 1) {
      const ff other(__shfl_down_sync(0xffffffffu, fs2.hi, o), __shfl_down_sync(0xffffffffu, fs2.lo, o));
      fs2 = fs2 + other;
      emax = fmaxf(emax, __shfl_down_sync(0xffffffffu, emax, o));
      qmin = fminf(qmin, __shfl_down_sync(0xffffffffu, qmin, o));
      qmax = fmaxf(qmax, __shfl_down_sync(0xffffffffu, qmax, o));
    }
    __shared__ float red[5][kDecThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = fs2.hi;
      red[1][wid] = fs2.lo;
      red[2][wid] = emax;
      red[3][wid] = qmin;
      red[4][wid] = qmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      ff a(0.f, 0.f);
      float b = 0.f, c = INFINITY, d = -INFINITY;
      for (int w = 0; w < kDecThreads / 32; ++w) {
        a = a + ff(red[0][w], red[1][w]);
        b = fmaxf(b, red[2][w]);
        c = fminf(c, red[3][w]);
        d = fmaxf(d, red[4][w]);
      }
      partials[4 * (long long)tile + 0] = (double)a.hi + (double)a.lo;
      partials[4 * (long long)tile + 1] = b;
      partials[4 * (long long)tile + 2] = c;
      partials[4 * (long long)tile + 3] = d;
    }
  }
}

template <int P, typename V>
size_t decode3d_smem(int ncx, int ncy, int ncz) {
  return dec_smem_layout(P + 1, ncx, ncy, ncz).total;
}

long long decode3d_tiles(const LayoutDev& L) {
  return ((L.M[0] + kDecTX - 1) / kDecTX) * ((L.M[1] + kDecTY - 1) / kDecTY) * ((L.M[2] + kDecTZ - 1) / kDecTZ);
}

// Bound on the control points a tile of `t` consecutive points touches.
static int tile_cps(const AxisDev& ax, int t) {
  // t points cover at most ceil((t-1) * nspans / (M-1)) + 1 spans
  const long long M = ax.M;
  if (M <= 1) return ax.p + 1;
  const long long spans = ((long long)(t - 1) * ax.nspans + (M - 2)) / (M - 1) + 1;
  return (int)std::min<long long>(spans + ax.p, ax.n);
}

template <typename V, typename TQ, typename TOut, bool RESID>
bool launch_decode3d(const LayoutDev& L, const V* P, const TQ* Q, TOut* out, double* partials, cudaStream_t st) {
  const int p = L.ax[0].p;
  if (L.dim != 3 || L.ax[1].p != p || L.ax[2].p != p) return false;
  const int ncx = tile_cps(L.ax[0], kDecTX), ncy = tile_cps(L.ax[1], kDecTY), ncz = tile_cps(L.ax[2], kDecTZ);
  const long long tiles = decode3d_tiles(L);
  const long long ntx = (L.M[0] + kDecTX - 1) / kDecTX, nty = (L.M[1] + kDecTY - 1) / kDecTY,
                  ntz = (L.M[2] + kDecTZ - 1) / kDecTZ;
  if (tiles > (1LL << 31) - 1 || ntx > INT32_MAX || nty > 65535 || ntz > 65535) return false;
  const dim3 grid((unsigned)ntx, (unsigned)nty, (unsigned)ntz);
  auto go = [&](auto kernel, size_t smem) {
    ensure_smem(kernel, smem);
    kernel<<<grid, kDecThreads, smem, st>>>(L, P, Q, out, partials);
  };
#define MFA_DEC_CASE(PP)                                                    \
  case PP: {                                                                \
    const size_t sm = decode3d_smem<PP, V>(ncx, ncy, ncz);                  \
    if (sm > 200 * 1024) return false;                                      \
    go(k_decode3d<PP, V, TQ, TOut, RESID>, sm);                             \
    return true;                                                            \
  }
  switch (p) {
    MFA_DEC_CASE(2)
    MFA_DEC_CASE(3)
    MFA_DEC_CASE(4)
    MFA_DEC_CASE(5)
    default:
      return false;
  }
#undef MFA_DEC_CASE
}

template bool launch_decode3d<ff, float, float, true>(const LayoutDev&, const ff*, const float*, float*, double*,
                                                      cudaStream_t);
template bool launch_decode3d<ff, double, float, true>(const LayoutDev&, const ff*, const double*, float*, double*,
                                                       cudaStream_t);
template bool launch_decode3d<ff, float, float, false>(const LayoutDev&, const ff*, const float*, float*, double*,
                                                       cudaStream_t);
template bool launch_decode3d<ff, float, double, false>(const LayoutDev&, const ff*, const float*, double*, double*,
                                                        cudaStream_t);

}  // namespace mfa

namespace mfa {

// ---------------------------------------------------------------------------
// Schwarz step k >= 1 as iterative refinement of every subdomain's own copy
// (Sec. 2.3.2; the Schur decoupling of Eq. global-system):
//   Z_s   = (X_s^{k-1} on U, P^{k-1} on the frame F)     the local spline
//   r_s   = B_U - A_L[U, :] Z_s                          float-float residual
//   X_s^k = X_s^{k-1} + (A_U,0 x A_U,1 x A_U,2)^{-1} r_s  FP32 correction
// In exact arithmetic X_s^k = A_U^{-1} (B_U - A_L[U, F] P_F^{k-1}), the
// constrained local solve.  The residual is taken against the subdomain's own
// previous copy, so it vanishes as the iteration converges and the FP32
// correction leaves no rounding floor (mixed-precision iterative refinement).
//
// One CTA per subdomain: Z_s streams through shared memory plane by plane
// along z (the next plane is fetched into registers while the current one is
// processed); per plane the x and y band products run in shared memory and the
// z band product accumulates in a register ring of 2P+1 owned z-points per
// owned (x, y) pair.  The residual box (FP32) stays in shared memory for the
// three fibre solves.
// ---------------------------------------------------------------------------

struct Step3dArgs {
  LayoutDev L;
  const long long* offL;
};

template <int P>
__device__ __forceinline__ void load_band_rows(const AxisDev& ax, const AxisSub& b, float* h, float* l) {
  // full band rows of A_L for the owned rows: row u holds A(oU+u, oU+u-P+e), e = 0..2P
  constexpr int B = 2 * P + 1;
  const double* A = ax.AL + (long long)b.bandL * (P + 1);
  for (int i = threadIdx.x; i < b.nU * B; i += blockDim.x) {
    const int u = i / B, e = i - u * B;
    const int r = b.oU + u, c = r - P + e;
    double v = 0.0;
    if (c >= 0 && c < b.nL) v = c >= r ? A[(long long)r * (P + 1) + (c - r)] : A[(long long)c * (P + 1) + (r - c)];
    const ff f(v);
    h[i] = f.hi;
    l[i] = f.lo;
  }
}

// In-place FP32 banded Cholesky solve of one fibre: L y = c, L^T x = y.
// F rows hold 1/L(i,i) at [i*W] and L(i,i-e) at [i*W+e].
template <int P>
__device__ __forceinline__ void solve_fibre(float* x, int n, int s, const float* F) {
  constexpr int W = P + 1;
  for (int i = 0; i < n; ++i) {
    float acc = x[i * s];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i - e >= 0) acc = fmaf(-F[i * W + e], x[(i - e) * s], acc);
    x[i * s] = acc * F[i * W];
  }
  for (int i = n - 1; i >= 0; --i) {
    float acc = x[i * s];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i + e < n) acc = fmaf(-F[(i + e) * W + e], x[(i + e) * s], acc);
    x[i * s] = acc * F[i * W];
  }
}

// The same solve in float-float (iteration 0 uses it on the ill-conditioned
// window blocks).
template <int P>
__device__ __forceinline__ void solve_fibre_ff(ff* x, int n, int s, const float* Fh, const float* Fl) {
  constexpr int W = P + 1;
  for (int i = 0; i < n; ++i) {
    ff acc = x[i * s];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i - e >= 0) AccFF::add_v(acc, -Fh[i * W + e], -Fl[i * W + e], x[(i - e) * s]);
    x[i * s] = AccFF::finish(acc) * ff(Fh[i * W], Fl[i * W]);
  }
  for (int i = n - 1; i >= 0; --i) {
    ff acc = x[i * s];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i + e < n) AccFF::add_v(acc, -Fh[(i + e) * W + e], -Fl[(i + e) * W + e], x[(i + e) * s]);
    x[i * s] = AccFF::finish(acc) * ff(Fh[i * W], Fl[i * W]);
  }
}

template <int P, int NT, int NPAIR, int NPRE>
__global__ void __launch_bounds__(NT, 2) k_schwarz3d_ff(Step3dArgs A, const ff* __restrict__ Pg,
                                                         const ff* __restrict__ BL, ff* __restrict__ X) {
  constexpr int W = P + 1, B = 2 * P + 1, NG = NT / 32, XR = 4;
  extern __shared__ __align__(128) unsigned char smem[];
  const LayoutDev& L = A.L;
  const int s = blockIdx.x;
  int s0, s1, s2;
  sub_pieces(L, s, s0, s1, s2);
  const AxisSub bx = L.ax[0].subs[s0], by = L.ax[1].subs[s1], bz = L.ax[2].subs[s2];
  const int nL0 = bx.nL, nL1 = by.nL, nL2 = bz.nL;
  const int nU0 = bx.nU, nU1 = by.nU, nU2 = bz.nU;
  const int oU0 = bx.oU, oU1 = by.oU, oU2 = bz.oU;
  const long long n0 = L.ncp[0], n01 = L.ncp[0] * L.ncp[1];
  // thread map: lanes along the owned x points (nU0 <= 32), groups over y
  const int ux = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const bool xin = ux < nU0;

  float* axh = reinterpret_cast<float*>(smem);  // [nU0][B]
  float* axl = axh + nU0 * B;
  float* ayh = axl + nU0 * B;                    // [nU1][B]
  float* ayl = ayh + nU1 * B;
  float* azh = ayl + nU1 * B;                    // [nU2][B]
  float* azl = azh + nU2 * B;
  float* fx = azl + nU2 * B;                     // [nU][W] FP32 factors of A_U per axis
  float* fy = fx + nU0 * W;
  float* fz = fy + nU1 * W;
  size_t off = (size_t)(2 * B * (nU0 + nU1 + nU2) + W * (nU0 + nU1 + nU2)) * 4;
  off = (off + 15) & ~size_t(15);
  // the plane and the x-band result carry P zero columns / rows on each side,
  // so the band products read without bounds checks (band entries outside L
  // are zero as well)
  const int ldp = nL0 + 2 * P;
  ff* Pp = reinterpret_cast<ff*>(smem + off);    // [nL1][P + nL0 + P]
  off += (size_t)nL1 * ldp * sizeof(ff);
  ff* Y1 = reinterpret_cast<ff*>(smem + off);    // [P + nL1 + P][nU0]
  off += (size_t)(nL1 + 2 * P) * nU0 * sizeof(ff);
  float* R = reinterpret_cast<float*>(smem + off);  // [nU2][nU1][nU0]

  load_band_rows<P>(L.ax[0], bx, axh, axl);
  load_band_rows<P>(L.ax[1], by, ayh, ayl);
  load_band_rows<P>(L.ax[2], bz, azh, azl);
  for (int i = threadIdx.x; i < nU0 * W; i += NT) fx[i] = L.ax[0].facU_f[(long long)bx.bandU * W + i];
  for (int i = threadIdx.x; i < nU1 * W; i += NT) fy[i] = L.ax[1].facU_f[(long long)by.bandU * W + i];
  for (int i = threadIdx.x; i < nU2 * W; i += NT) fz[i] = L.ax[2].facU_f[(long long)bz.bandU * W + i];

  const int nplane = nL1 * nL0;
  for (int i = threadIdx.x; i < nL1 * 2 * P; i += NT) {
    const int ly = i / (2 * P), e = i - ly * 2 * P;
    Pp[ly * ldp + (e < P ? e : nL0 + e)] = ff(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < 2 * P * nU0; i += NT) {
    const int r = i / nU0, x = i - r * nU0;
    Y1[(r < P ? r : nL1 + r) * nU0 + x] = ff(0.f, 0.f);
  }
  int pdst[NPRE];  // where this thread's prefetched values land in the padded plane
#pragma unroll
  for (int k = 0; k < NPRE; ++k) {
    const int i = threadIdx.x + k * NT;
    const int ly = i / nL0, lx = i - ly * nL0;
    pdst[k] = i < nplane ? ly * ldp + P + lx : -1;
  }
  ff ring[NPAIR][B];  // pair i of this thread: owned (ux, uy = grp + NG*i)
#pragma unroll
  for (int i = 0; i < NPAIR; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) ring[i][j] = ff(0.f, 0.f);
  const ff* bl = BL + A.offL[s];
  ff* xs = X + A.offL[s];
  const ff* pg = Pg + (long long)bx.l0 + n0 * by.l0 + n01 * bz.l0;

  // planes that reach an owned z-point through the band
  const int lz_lo = max(0, oU2 - P), lz_hi = min(nL2 - 1, oU2 + nU2 - 1 + P);
  ff pre[NPRE];
  auto fetch = [&](int lz) {
    const bool zin = lz >= oU2 && lz < oU2 + nU2;
#pragma unroll
    for (int k = 0; k < NPRE; ++k) {
      const int i = threadIdx.x + k * NT;
      if (i < nplane) {
        const int ly = i / nL0, lx = i - ly * nL0;
        const bool own = zin && ly >= oU1 && ly < oU1 + nU1 && lx >= oU0 && lx < oU0 + nU0;
        pre[k] = own ? xs[(long long)lz * nplane + i] : pg[lx + n0 * ly + n01 * lz];
      }
    }
  };
  auto b_at = [&](int i, int uz) -> ff {
    const int uy = grp + NG * i;
    if (!xin || uy >= nU1 || uz < 0 || uz >= nU2) return ff(0.f, 0.f);
    return bl[(oU0 + ux) + (long long)nL0 * ((oU1 + uy) + (long long)nL1 * (oU2 + uz))];
  };
  auto write_resid = [&](int i, int uz, ff b) {
    const int uy = grp + NG * i;
    const ff r = b - AccFF::finish(ring[i][0]);
    R[(uz * nU1 + uy) * nU0 + ux] = r.hi + r.lo;
  };
  // B_U of the owned z-point that completes at the current plane, fetched one plane ahead
  ff bnext[NPAIR];
#pragma unroll
  for (int i = 0; i < NPAIR; ++i) bnext[i] = b_at(i, lz_lo - oU2 - P);
  fetch(lz_lo);
  for (int lz = lz_lo; lz <= lz_hi; ++lz) {
#pragma unroll
    for (int k = 0; k < NPRE; ++k)
      if (pdst[k] >= 0) Pp[pdst[k]] = pre[k];
    __syncthreads();
    if (lz < lz_hi) fetch(lz + 1);
    // x band product, owned x rows; XR independent rows per thread in flight
    if (xin) {
      const int c0 = oU0 + ux - P;
      for (int ly0 = grp; ly0 < nL1; ly0 += XR * NG) {
        ff acc[XR];
#pragma unroll
        for (int k = 0; k < XR; ++k) acc[k] = ff(0.f, 0.f);
        const ff* prow = Pp + P + c0;
#pragma unroll
        for (int e = 0; e < B; ++e) {
          const float h = axh[ux * B + e], l = axl[ux * B + e];
#pragma unroll
          for (int k = 0; k < XR; ++k) {
            const int ly = ly0 + k * NG;
            if (ly < nL1) AccFF::add_v(acc[k], h, l, prow[ly * ldp + e]);
          }
        }
#pragma unroll
        for (int k = 0; k < XR; ++k) {
          const int ly = ly0 + k * NG;
          if (ly < nL1) Y1[(P + ly) * nU0 + ux] = AccFF::finish(acc[k]);
        }
      }
    }
    __syncthreads();
    // y band product, owned y rows; each result feeds only this thread's own
    // z ring, so it stays in registers
    ff y2r[NPAIR];
#pragma unroll
    for (int i = 0; i < NPAIR; ++i) {
      const int uy = grp + NG * i;
      y2r[i] = ff(0.f, 0.f);
      if (xin && uy < nU1) {
        const int c0 = oU1 + uy - P;
        ff acc(0.f, 0.f);
        const ff* ycol = Y1 + (P + c0) * nU0 + ux;
#pragma unroll
        for (int e = 0; e < B; ++e) AccFF::add_v(acc, ayh[uy * B + e], ayl[uy * B + e], ycol[e * nU0]);
        y2r[i] = AccFF::finish(acc);
      }
    }
    // z band product into the ring: slot j holds owned z-point uz = lz - oU2 - P + j
    const int uzb = lz - oU2 - P;
    ff bcur[NPAIR];
#pragma unroll
    for (int i = 0; i < NPAIR; ++i) {
      bcur[i] = bnext[i];
      bnext[i] = b_at(i, uzb + 1);
    }
#pragma unroll
    for (int i = 0; i < NPAIR; ++i) {
      const int uy = grp + NG * i;
      if (xin && uy < nU1) {
        const ff y2 = y2r[i];
#pragma unroll
        for (int j = 0; j < B; ++j) {
          const int uz = uzb + j;
          if (uz >= 0 && uz < nU2) AccFF::add_v(ring[i][j], azh[uz * B + (2 * P - j)], azl[uz * B + (2 * P - j)], y2);
        }
        if (uzb >= 0 && uzb < nU2) write_resid(i, uzb, bcur[i]);  // slot 0 is complete
      }
#pragma unroll
      for (int j = 0; j < B - 1; ++j) ring[i][j] = ring[i][j + 1];
      ring[i][B - 1] = ff(0.f, 0.f);
    }
    // no barrier: the next plane's stores to Pp follow the x-band barrier of
    // this plane (every thread has finished reading Pp), and Y1 is rewritten
    // only after the next plane's first barrier (every thread has finished
    // its y band here)
  }
  // owned z-points whose band ended with the last plane
  {
    const int uzb = lz_hi + 1 - oU2 - P;  // z-point now in slot 0
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int uz = uzb + j;
#pragma unroll
      for (int i = 0; i < NPAIR; ++i) {
        const int uy = grp + NG * i;
        if (xin && uy < nU1 && uz >= 0 && uz < nU2) write_resid(i, uz, b_at(i, uz));
      }
#pragma unroll
      for (int i = 0; i < NPAIR; ++i) {
#pragma unroll
        for (int jj = 0; jj < B - 1; ++jj) ring[i][jj] = ring[i][jj + 1];
        ring[i][B - 1] = ff(0.f, 0.f);
      }
    }
  }
  __syncthreads();
  // correction c = A_U^{-1} r in FP32, one fibre per thread and axis
  for (int f = threadIdx.x; f < nU1 * nU2; f += NT) solve_fibre<P>(R + f * nU0, nU0, 1, fx);
  __syncthreads();
  for (int f = threadIdx.x; f < nU0 * nU2; f += NT) {
    const int fx0 = f % nU0, uz = f / nU0;
    solve_fibre<P>(R + uz * nU1 * nU0 + fx0, nU1, nU0, fy);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < nU0 * nU1; f += NT) solve_fibre<P>(R + f, nU2, nU0 * nU1, fz);
  __syncthreads();
  // refined copy X_s^k = X_s^{k-1} + c_s (four z-planes of loads in flight)
  if (xin) {
#pragma unroll
    for (int i = 0; i < NPAIR; ++i) {
      const int uy = grp + NG * i;
      if (uy >= nU1) continue;
      for (int uz0 = 0; uz0 < nU2; uz0 += 4) {
        ff v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int uz = uz0 + t;
          if (uz < nU2) v[t] = xs[(oU0 + ux) + (long long)nL0 * ((oU1 + uy) + (long long)nL1 * (oU2 + uz))];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int uz = uz0 + t;
          if (uz < nU2)
            xs[(oU0 + ux) + (long long)nL0 * ((oU1 + uy) + (long long)nL1 * (oU2 + uz))] =
                v[t] + ff(R[(uz * nU1 + uy) * nU0 + ux]);
        }
      }
    }
  }
}

template <int P>
size_t step3d_smem(int nL0, int nL1, int nU0, int nU1, int nU2) {
  constexpr int W = P + 1, B = 2 * P + 1;
  size_t off = (size_t)(2 * B * (nU0 + nU1 + nU2) + W * (nU0 + nU1 + nU2)) * 4;
  off = (off + 15) & ~size_t(15);
  off += (size_t)nL1 * (nL0 + 2 * P) * sizeof(ff) + (size_t)(nL1 + 2 * P) * nU0 * sizeof(ff);
  off += (size_t)nU0 * nU1 * nU2 * sizeof(float);
  return off;
}

constexpr int kStepThreads = 256;

bool launch_schwarz3d_ff(const LayoutDev& L, const long long* offL, const int* maxnL, const int* maxnU, const ff* P,
                         const ff* BL, ff* X, cudaStream_t st) {
  const int p = L.ax[0].p;
  if (L.dim != 3 || L.ax[1].p != p || L.ax[2].p != p) return false;
  Step3dArgs A;
  A.L = L;
  A.offL = offL;
  constexpr int NG = kStepThreads / 32;
  const int nplane = maxnL[0] * maxnL[1];
  // owned x points on the lanes, owned y points on NPAIR rounds of the groups
  if (maxnU[0] > 32 || maxnU[1] > 4 * NG || nplane > 4 * kStepThreads) return false;
  auto go = [&](auto kernel, size_t sm) {
    ensure_smem(kernel, sm, true);
    kernel<<<L.nsub, kStepThreads, sm, st>>>(A, P, BL, X);
  };
#define MFA_STEP_CASE(PP)                                                                      \
  case PP: {                                                                                   \
    const size_t sm = step3d_smem<PP>(maxnL[0], maxnL[1], maxnU[0], maxnU[1], maxnU[2]);       \
    if (sm > 220 * 1024) return false;                                                         \
    if (maxnU[1] <= 2 * NG)                                                                    \
      go(k_schwarz3d_ff<PP, kStepThreads, 2, 4>, sm);                                          \
    else                                                                                       \
      go(k_schwarz3d_ff<PP, kStepThreads, 4, 4>, sm);                                          \
    return true;                                                                               \
  }
  switch (p) {
    MFA_STEP_CASE(2)
    MFA_STEP_CASE(3)
    MFA_STEP_CASE(4)
    MFA_STEP_CASE(5)
    default:
      return false;
  }
#undef MFA_STEP_CASE
}

// ---------------------------------------------------------------------------
// Update (Sec. 2.3.2) in float-float: P^k(g) = (1/n_s) sum of the owned copies
// of g in a fixed order; metrics max|P^k - P^{k-1}|, max|P^k| and the copy
// spread are formed from float-float differences, so no FP64 arithmetic runs.
// One launch, two kinds of block:
//   - block s < nsub copies the box of control points that subdomain s owns
//     alone on every axis (P = its copy): rows of the box stream from the copy
//     to P, lanes along x, four rows in flight per warp;
//   - the other blocks take the control points with two owners on some axis,
//     rows handed out by an atomic counter: rows with two owners along y or z
//     in full, the other rows at the x positions with two owners.  Every copy
//     of such a point is loaded independently before they are combined; the
//     owner and offset tables sit in shared memory.
// ---------------------------------------------------------------------------

// 1/n as float-float, n = 1..8 (hi = 1/n rounded to FP32, lo = the rest
// rounded), fixed when the module loads so a reloaded module has them too
#define MFA_INV_HI(n) ((float)(1.0 / (n)))
#define MFA_INV_LO(n) ((float)(1.0 / (n) - (double)MFA_INV_HI(n)))
__constant__ float c_inv_hi[9] = {0.f,           MFA_INV_HI(1), MFA_INV_HI(2), MFA_INV_HI(3), MFA_INV_HI(4),
                                  MFA_INV_HI(5), MFA_INV_HI(6), MFA_INV_HI(7), MFA_INV_HI(8)};
__constant__ float c_inv_lo[9] = {0.f,           MFA_INV_LO(1), MFA_INV_LO(2), MFA_INV_LO(3), MFA_INV_LO(4),
                                  MFA_INV_LO(5), MFA_INV_LO(6), MFA_INV_LO(7), MFA_INV_LO(8)};
#undef MFA_INV_HI
#undef MFA_INV_LO
constexpr int kAvgThreads = 256;

// Tables of the update kept in shared memory when they fit (else read from
// global memory): owner entries of every axis, L sizes, copy offsets.
struct AvgTabs {
  const int4 *ot0, *ot1, *ot2;
  const int *nl0, *nl1;
  const long long* off;
  const int *pk0, *pk1, *pk2;  // owner-takes: slot (0 / 1) of the Greville owner per axis
};

// All copies of control point (g0, g1, g2), loaded independently: slot
// c = c0 + 2 c1 + 4 c2 picks owner c_a along axis a.
struct AvgCopies {
  ff v[8];
  unsigned ok;
  ff prev;
};

__device__ __forceinline__ void avg_load(const LayoutDev& L, const AvgTabs& T, const ff* __restrict__ X,
                                         const ff* __restrict__ Pprev, long long g, int4 o0, int4 o1, int4 o2,
                                         AvgCopies& cp) {
  cp.prev = Pprev ? Pprev[g] : ff(0.f, 0.f);
  cp.ok = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int c0 = c & 1, c1 = (c >> 1) & 1, c2 = c >> 2;
    const int sa0 = c0 ? o0.z : o0.x, li0 = c0 ? o0.w : o0.y;
    const int sa1 = c1 ? o1.z : o1.x, li1 = c1 ? o1.w : o1.y;
    const int sa2 = c2 ? o2.z : o2.x, li2 = c2 ? o2.w : o2.y;
    const bool ok = sa0 >= 0 && sa1 >= 0 && sa2 >= 0;
    cp.v[c] = ff(0.f, 0.f);
    if (ok) {
      const int s = sa0 + L.S[0] * (sa1 + L.S[1] * sa2);
      const long long li = li0 + (long long)T.nl0[sa0] * (li1 + (long long)T.nl1[sa1] * li2);
      cp.v[c] = X[T.off[s] + li];
      cp.ok |= 1u << c;
    }
  }
}

__device__ __forceinline__ void avg_finish(const AvgCopies& cp, bool has_prev, long long g, ff* __restrict__ P,
                                           float& dmax, float& pmax, float& spread, int owner_slot) {
  ff sum(0.f, 0.f), first(0.f, 0.f);
  float dlo = 0.f, dhi = 0.f;
  int cnt = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (!(cp.ok & (1u << c))) continue;
    if (cnt == 0) {
      sum = cp.v[c];
      first = cp.v[c];
    } else {
      sum = sum + cp.v[c];
      const ff d = cp.v[c] - first;
      const float df = d.hi + d.lo;
      dlo = fminf(dlo, df);
      dhi = fmaxf(dhi, df);
    }
    ++cnt;
  }
  ff pn = cnt == 1 ? sum : sum * ff(c_inv_hi[cnt], c_inv_lo[cnt]);
  if (owner_slot >= 0) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c == owner_slot) pn = cp.v[c];
  }
  P[g] = pn;
  pmax = fmaxf(pmax, fabsf(pn.hi));
  spread = fmaxf(spread, dhi - dlo);
  if (has_prev) {
    const ff d = pn - cp.prev;
    dmax = fmaxf(dmax, fabsf(d.hi + d.lo));
  }
}

// Metrics of one control point with a single copy v (P = v).
__device__ __forceinline__ void avg_single(ff v, const ff* __restrict__ Pprev, long long g, ff* __restrict__ P,
                                           float& dmax, float& pmax) {
  P[g] = v;
  pmax = fmaxf(pmax, fabsf(v.hi));
  if (Pprev) {
    const ff d = v - Pprev[g];
    dmax = fmaxf(dmax, fabsf(d.hi + d.lo));
  }
}

__global__ void __launch_bounds__(kAvgThreads, 3) k_average_ff(LayoutDev L, const long long* __restrict__ offL,
                                                               const ff* __restrict__ X, ff* __restrict__ P,
                                                               const ff* __restrict__ Pprev, float* __restrict__ part,
                                                               unsigned* __restrict__ row_ctr,
                                                               unsigned long long* __restrict__ metrics,
                                                               int stage_tables, int rule) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n0 = (int)L.ncp[0], n1 = (int)L.ncp[1], n2 = (int)L.ncp[2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float dmax = 0.f, pmax = 0.f, spread = 0.f;
  if ((int)blockIdx.x < L.nsub) {
    // ---- the single-owner box of subdomain s
    const int s = blockIdx.x;
    int s0, s1, s2;
    sub_pieces(L, s, s0, s1, s2);
    const int2 r0 = L.ax[0].one_rng[s0], r1 = L.ax[1].one_rng[s1], r2 = L.ax[2].one_rng[s2];
    const AxisSub b0 = L.ax[0].subs[s0], b1 = L.ax[1].subs[s1], b2 = L.ax[2].subs[s2];
    const int nx = r0.y - r0.x, ny = r1.y - r1.x, nrows = ny * (r2.y - r2.x);
    const ff* xs = X + offL[s] + (r0.x - b0.l0);
    ff* ps = P + r0.x;
    const ff* qs = Pprev ? Pprev + r0.x : nullptr;
    const int nw = blockDim.x >> 5;
    for (int rb = wid; rb < nrows; rb += 4 * nw) {
      long long xo[4], po[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = min(rb + u * nw, nrows - 1);
        const int y = r % ny, z = r / ny;
        xo[u] = (long long)b0.nL * ((r1.x + y - b1.l0) + (long long)b1.nL * (r2.x + z - b2.l0));
        po[u] = (long long)n0 * ((r1.x + y) + (long long)n1 * (r2.x + z));
      }
      for (int x = lane; x < nx; x += 32) {
        ff v[4], q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[u] = xs[xo[u] + x];
          q[u] = qs ? qs[po[u] + x] : ff(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (rb + u * nw >= nrows) continue;
          ps[po[u] + x] = v[u];
          pmax = fmaxf(pmax, fabsf(v[u].hi));
          if (qs) {
            const ff d = v[u] - q[u];
            dmax = fmaxf(dmax, fabsf(d.hi + d.lo));
          }
        }
      }
    }
  } else {
    // ---- control points with two owners on some axis
    AvgTabs T{L.ax[0].own_tab, L.ax[1].own_tab, L.ax[2].own_tab, L.ax[0].nL_tab, L.ax[1].nL_tab, offL,
              L.ax[0].own_pick, L.ax[1].own_pick, L.ax[2].own_pick};
    if (stage_tables) {
      int4* t0 = reinterpret_cast<int4*>(smem);
      int4* t1 = t0 + n0;
      int4* t2 = t1 + n1;
      long long* off = reinterpret_cast<long long*>(t2 + n2);
      int* l0 = reinterpret_cast<int*>(off + L.nsub);
      int* l1 = l0 + L.S[0];
      int* k0 = l1 + L.S[1];
      int* k1 = k0 + n0;
      int* k2 = k1 + n1;
      for (int i = threadIdx.x; i < n0; i += blockDim.x) t0[i] = T.ot0[i];
      for (int i = threadIdx.x; i < n1; i += blockDim.x) t1[i] = T.ot1[i];
      for (int i = threadIdx.x; i < n2; i += blockDim.x) t2[i] = T.ot2[i];
      for (int i = threadIdx.x; i < L.nsub; i += blockDim.x) off[i] = offL[i];
      for (int i = threadIdx.x; i < L.S[0]; i += blockDim.x) l0[i] = T.nl0[i];
      for (int i = threadIdx.x; i < L.S[1]; i += blockDim.x) l1[i] = T.nl1[i];
      for (int i = threadIdx.x; i < n0; i += blockDim.x) k0[i] = T.pk0[i];
      for (int i = threadIdx.x; i < n1; i += blockDim.x) k1[i] = T.pk1[i];
      for (int i = threadIdx.x; i < n2; i += blockDim.x) k2[i] = T.pk2[i];
      __syncthreads();
      T = AvgTabs{t0, t1, t2, l0, l1, off, k0, k1, k2};
    }
    const int nrows = L.n_full_rows + L.n_part_rows;
    constexpr int kChunk = 2;  // rows per grab
    for (;;) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(row_ctr, kChunk);
      base = __shfl_sync(0xffffffffu, base, 0);
      if ((int)base >= nrows) break;
      for (int k = (int)base; k < min((int)base + kChunk, nrows); ++k) {
        const int r = L.shared_rows[k];
        const int g1 = r % n1, g2 = r / n1;
        const int4 o1 = T.ot1[g1], o2 = T.ot2[g2];
        const bool full = k < L.n_full_rows;
        const int cnt = full ? n0 : L.n_shared_x;
        for (int j = lane; j < cnt; j += 32) {
          const int g0 = full ? j : L.shared_x[j];
          const long long g = (long long)g0 + (long long)n0 * r;
          AvgCopies cp;
          avg_load(L, T, X, Pprev, g, T.ot0[g0], o1, o2, cp);
          const int slot = rule == UPDATE_OWNER ? T.pk0[g0] + 2 * T.pk1[g1] + 4 * T.pk2[g2] : -1;
          avg_finish(cp, Pprev != nullptr, g, P, dmax, pmax, spread, slot);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
    pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    spread = fmaxf(spread, __shfl_down_sync(0xffffffffu, spread, o));
  }
  __shared__ float red[3][kAvgThreads / 32];
  if (lane == 0) {
    red[0][wid] = dmax;
    red[1][wid] = pmax;
    red[2][wid] = spread;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = red[0][0], b = red[1][0], c = red[2][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = fmaxf(a, red[0][w]);
      b = fmaxf(b, red[1][w]);
      c = fmaxf(c, red[2][w]);
    }
    part[3 * blockIdx.x + 0] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
  // the last block to finish reduces every block's partials, in a fixed
  // order, into metrics[0..2] (bit patterns of non-negative doubles)
  __shared__ int last_block;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last_block = atomicAdd(row_ctr + 1, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last_block) {
    __threadfence();
    float a = 0.f, b = 0.f, c = 0.f;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
      a = fmaxf(a, __ldcg(part + 3 * i));
      b = fmaxf(b, __ldcg(part + 3 * i + 1));
      c = fmaxf(c, __ldcg(part + 3 * i + 2));
    }
    for (int o = 16; o > 0; o >>= 1) {
      a = fmaxf(a, __shfl_down_sync(0xffffffffu, a, o));
      b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, o));
      c = fmaxf(c, __shfl_down_sync(0xffffffffu, c, o));
    }
    if (lane == 0) {
      red[0][wid] = a;
      red[1][wid] = b;
      red[2][wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        a = fmaxf(a, red[0][w]);
        b = fmaxf(b, red[1][w]);
        c = fmaxf(c, red[2][w]);
      }
      metrics[0] = (unsigned long long)__double_as_longlong((double)a);
      metrics[1] = (unsigned long long)__double_as_longlong((double)b);
      metrics[2] = (unsigned long long)__double_as_longlong((double)c);
    }
  }
}

long long average_ff_blocks(const LayoutDev& L) {
  const int list = 3 * device_sm_count();  // blocks on the shared control points: 3 per SM
  return L.nsub + (list < kAvgListBlocks ? list : kAvgListBlocks);
}

// `part` holds 3 floats per block of the launch (average_ff_blocks) and, after
// them, the row counter of the shared control points and the finished-block
// counter.
void launch_average_ff(const LayoutDev& L, const long long* offL, const ff* X, ff* P, const ff* Pprev, float* part,
                       unsigned long long* metrics, cudaStream_t st, int rule) {
  const size_t tab = (size_t)(L.ncp[0] + L.ncp[1] + L.ncp[2]) * (sizeof(int4) + sizeof(int)) +
                     (size_t)L.nsub * sizeof(long long) + (size_t)(L.S[0] + L.S[1]) * sizeof(int);
  const int stage = tab <= 40 * 1024;
  const long long nblk = average_ff_blocks(L);
  unsigned* row_ctr = reinterpret_cast<unsigned*>(part + 3 * nblk);
  cudaMemsetAsync(row_ctr, 0, 2 * sizeof(unsigned), st);
  k_average_ff<<<(unsigned)nblk, kAvgThreads, stage ? tab : 0, st>>>(L, offL, X, P, Pprev, part, row_ctr, metrics,
                                                                      stage, rule);
}

}  // namespace mfa

namespace mfa {

// ---------------------------------------------------------------------------
// Iteration 0 (Algorithm 1: decoupled unconstrained local solves):
// X_s = (A_L,0 x A_L,1 x A_L,2)^{-1} B_L in float-float.  Pass 1 solves the x
// and y fibres of one z-plane of one subdomain in shared memory; pass 2 solves
// the z fibres in place, one fibre per thread (coalesced across x).
// ---------------------------------------------------------------------------

constexpr int kIt0Planes = 4;

template <int P>
__global__ void __launch_bounds__(128) k_iter0_xy_ff(LayoutDev L, const long long* __restrict__ offL,
                                                     const ff* __restrict__ BL, ff* __restrict__ X) {
  constexpr int W = P + 1;
  extern __shared__ __align__(128) unsigned char smem[];
  const int s = blockIdx.x, lz0 = blockIdx.y * kIt0Planes;
  int s0, s1, s2;
  sub_pieces(L, s, s0, s1, s2);
  const AxisSub bx = L.ax[0].subs[s0], by = L.ax[1].subs[s1], bz = L.ax[2].subs[s2];
  if (lz0 >= bz.nL) return;
  const int npl = min(kIt0Planes, bz.nL - lz0);
  const int nL0 = bx.nL, nL1 = by.nL;
  float* fxh = reinterpret_cast<float*>(smem);
  float* fxl = fxh + nL0 * W;
  float* fyh = fxl + nL0 * W;
  float* fyl = fyh + nL1 * W;
  size_t off = (size_t)2 * W * (nL0 + nL1) * 4;
  off = (off + 15) & ~size_t(15);
  ff* T = reinterpret_cast<ff*>(smem + off);  // [npl][nL1][nL0]
  const int npp = nL0 * nL1;
  const long long base = offL[s] + (long long)lz0 * npp;
  // the planes' right-hand sides as asynchronous 8-byte copies, all in
  // flight together, under the factor tables' loads
  for (int i = threadIdx.x; i < npl * npp; i += blockDim.x) cp_async_8(T + i, BL + base + i);
  cp_async_commit();
  const ff* Fx = L.ax[0].facL_ff + (long long)bx.bandL * W;
  const ff* Fy = L.ax[1].facL_ff + (long long)by.bandL * W;
  for (int i = threadIdx.x; i < nL0 * W; i += blockDim.x) {
    fxh[i] = Fx[i].hi;
    fxl[i] = Fx[i].lo;
  }
  for (int i = threadIdx.x; i < nL1 * W; i += blockDim.x) {
    fyh[i] = Fy[i].hi;
    fyl[i] = Fy[i].lo;
  }
  cp_async_wait_all();
  __syncthreads();
  for (int f = threadIdx.x; f < npl * nL1; f += blockDim.x) solve_fibre_ff<P>(T + f * nL0, nL0, 1, fxh, fxl);
  __syncthreads();
  for (int f = threadIdx.x; f < npl * nL0; f += blockDim.x) {
    const int pl = f / nL0, x = f - pl * nL0;
    solve_fibre_ff<P>(T + pl * npp + x, nL1, nL0, fyh, fyl);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npl * npp; i += blockDim.x) X[base + i] = T[i];
}

template <int P>
__global__ void __launch_bounds__(128) k_iter0_z_ff(LayoutDev L, const long long* __restrict__ offL,
                                                    ff* __restrict__ X) {
  constexpr int W = P + 1;
  const int s = blockIdx.y;
  int s0, s1, s2;
  sub_pieces(L, s, s0, s1, s2);
  const AxisSub bx = L.ax[0].subs[s0], by = L.ax[1].subs[s1], bz = L.ax[2].subs[s2];
  const int nf = bx.nL * by.nL;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  const int n = bz.nL;
  const long long st = nf;
  ff* x = X + offL[s] + f;
  const ff* F = L.ax[2].facL_ff + (long long)bz.bandL * W;
  ff win[P];  // the last P solved values, win[0] the most recent
#pragma unroll
  for (int e = 0; e < P; ++e) win[e] = ff(0.f, 0.f);
  for (int i = 0; i < n; ++i) {
    ff acc = x[i * st];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i - e >= 0) {
        const ff Fe = F[i * W + e];
        AccFF::add_v(acc, -Fe.hi, -Fe.lo, win[e - 1]);
      }
    const ff y = AccFF::finish(acc) * F[i * W];
    x[i * st] = y;
#pragma unroll
    for (int e = P - 1; e > 0; --e) win[e] = win[e - 1];
    win[0] = y;
  }
#pragma unroll
  for (int e = 0; e < P; ++e) win[e] = ff(0.f, 0.f);
  for (int i = n - 1; i >= 0; --i) {
    ff acc = x[i * st];
#pragma unroll
    for (int e = 1; e <= P; ++e)
      if (i + e < n) {
        const ff Fe = F[(i + e) * W + e];
        AccFF::add_v(acc, -Fe.hi, -Fe.lo, win[e - 1]);
      }
    const ff v = AccFF::finish(acc) * F[i * W];
    x[i * st] = v;
#pragma unroll
    for (int e = P - 1; e > 0; --e) win[e] = win[e - 1];
    win[0] = v;
  }
}

// Returns the number of kernels launched (0 when not covered).
int launch_iter0_3d_ff(const LayoutDev& L, const long long* offL, const int* maxnL, const ff* BL, ff* X,
                       cudaStream_t st) {
  const int p = L.ax[0].p;
  if (L.dim != 3 || L.ax[1].p != p || L.ax[2].p != p) return 0;
  const size_t smem = (((size_t)2 * (p + 1) * (maxnL[0] + maxnL[1]) * 4 + 15) & ~size_t(15)) +
                      (size_t)kIt0Planes * maxnL[0] * maxnL[1] * sizeof(ff);
  if (smem > 200 * 1024) return 0;
  dim3 g1(L.nsub, (maxnL[2] + kIt0Planes - 1) / kIt0Planes);
  dim3 g2((maxnL[0] * maxnL[1] + 127) / 128, L.nsub);
  auto go = [&](auto kxy, auto kz) {
    ensure_smem(kxy, smem);
    kxy<<<g1, 128, smem, st>>>(L, offL, BL, X);
    kz<<<g2, 128, 0, st>>>(L, offL, X);
  };
  switch (p) {
    case 2: go(k_iter0_xy_ff<2>, k_iter0_z_ff<2>); return 2;
    case 3: go(k_iter0_xy_ff<3>, k_iter0_z_ff<3>); return 2;
    case 4: go(k_iter0_xy_ff<4>, k_iter0_z_ff<4>); return 2;
    case 5: go(k_iter0_xy_ff<5>, k_iter0_z_ff<5>); return 2;
    default: return 0;
  }
}

}  // namespace mfa

namespace mfa {

void ensure_smem_attr(const void* kernel, size_t bytes, bool carveout) {
  // the limit the kernel has in the current context right now (a context
  // created again after a reset starts from the default), only ever raised:
  // host threads launching the same kernel with different sizes (the
  // server's workers) check and raise it one at a time, so no thread lowers
  // the limit another thread's launch relies on
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    fa.maxDynamicSharedSizeBytes = 0;
    fa.preferredShmemCarveout = -1;
  }
  if ((size_t)fa.maxDynamicSharedSizeBytes < bytes &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    cudaGetLastError();  // the launch reports the problem
  if (carveout && fa.preferredShmemCarveout != 100 &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
    cudaGetLastError();
}

}  // namespace mfa

