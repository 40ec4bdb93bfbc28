// Internal declarations of the MFA library: device layout tables, batched
// per-subdomain tensor views and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ff.cuh"
#include "mfa.h"

namespace mfa {

// One subdomain along one grid axis (Sec. 2.2, Eq. vecp-layout):
//   core spans [a, b), window spans [w0, w1) = core + overlap per interior side,
//   data points [k0, k0 + m) with parameter in the closed window interval,
//   L = [l0, l0 + nL) control points touching the window,
//   U = [l0 + oU, l0 + oU + nU) owned control points (support meets the core).
struct AxisSub {
  int a, b, w0, w1;
  int k0, m;
  int l0, nL;
  int oU, nU;
  int bandL;  // first row of this piece in the per-axis L band arrays
  int bandU;  // first row of this piece in the per-axis U band arrays
};

// Knot layout of an axis.
enum { KMODE_FLOATING = 0, KMODE_CLAMPED = 2 };

// Per-axis device tables.  Spans are numbered by the first control point
// nonzero on them (span j has control points j .. j+p), so `nspans` counts
// span numbers, including numbers no span uses (between the pieces of a batch
// or across the repeated knots of a clamped interface); `gspans` is the
// number of knot spans of the axis's own grid.
struct AxisDev {
  int M, nspans, p, n, S;
  int pieces;               // 1: every piece (subs[i]) has its own knot vector with w1 - w0 spans over its
                            // own points, spans numbered from its l0 (a batch of independent fits)
  int kmode;                // KMODE_FLOATING, or KMODE_CLAMPED: interface knots repeated p times, so the
                            // points of core [a, b) use that core's own clamped uniform knots (b - a spans),
                            // spans numbered from the core's first owned control point
  int gspans;               // knot spans of the grid (uniform breakpoints i / gspans)
  const double* wts;        // [n] NURBS control-point weights, or nullptr (W = 1)
  const int* span;          // [M] knot span of every data point
  const double* vals_d;     // [M * (p+1)] N_{span+r,p}(u_k), r = 0..p
  const float* vals_f;      // same, rounded to FP32
  const ff* vals_ff;        // same, as float-float pairs
  const int* span_start;    // [nspans + 1] first point whose span is >= j
  const AxisSub* subs;      // [S]
  const int* own_first;     // [n] first subdomain-axis index owning CP g
  const int* own_count;     // [n] number of owners (1 or 2)
  const int4* own_tab;      // [n] {first owner, g - l0 in it, second owner or -1, g - l0 in it}
  const int* own_pick;      // [n] 0 or 1: which owner holds the Greville abscissa (owner-takes update)
  const int* nL_tab;        // [S] L size of every piece
  const int2* one_rng;      // [S] control points owned by piece i alone: [x, y) (contiguous)
  const double* AL;         // Gram band rows of every piece, upper storage: A(i, i+e) at [i*(p+1)+e]
  const double* facL_d;     // Cholesky band of A_L: [i*(p+1)] = 1/L(i,i), [i*(p+1)+e] = L(i,i-e)
  const float* facL_f;
  const ff* facL_ff;
  const double* facU_d;     // Cholesky band of A_U (owned rows only)
  const float* facU_f;
  const ff* facU_ff;
};

struct LayoutDev {
  int dim;
  int nsub;
  int S[3];
  long long ncp[3];    // n_a (1 for axes >= dim)
  long long M[3];
  AxisDev ax[3];
  int diag;            // 1: subdomain s uses piece s on every axis with more than one piece (a batch of
                       // independent fits); 0: the tensor product, s = s0 + S0 (s1 + S1 s2)
  // control points with two owners on some axis, by rows along x (row
  // r = g1 + n1 g2): `shared_rows` lists first the rows with two owners along
  // y or z (every x), then the others (only the x positions `shared_x`)
  const int* shared_rows;
  int n_full_rows, n_part_rows;
  const int* shared_x;
  int n_shared_x;
};

// The piece of subdomain s along each axis.
__host__ __device__ inline void sub_pieces(const LayoutDev& L, int s, int& s0, int& s1, int& s2) {
  if (L.diag) {
    s0 = L.S[0] > 1 ? s : 0;
    s1 = L.S[1] > 1 ? s : 0;
    s2 = L.S[2] > 1 ? s : 0;
  } else {
    s0 = s % L.S[0];
    s1 = (s / L.S[0]) % L.S[1];
    s2 = s / (L.S[0] * L.S[1]);
  }
}

// A strided 3-D view: element (i0,i1,i2) at off + i0*st[0] + i1*st[1] + i2*st[2].
struct View {
  long long off;
  long long st[3];
  int n[3];
};

// One subdomain's operand description for an operation along one axis.
struct AxisOp {
  View in, out;
  int k0;    // global index of point 0 on the point-indexed side of the axis
  int kend;  // one past the last point that may contribute (contract)
  int c0;    // global index of CP 0 on the CP-indexed side of the axis
  int sa;    // subdomain-axis index along the op axis
  int oU;    // row offset of the output inside L (band apply), 0 otherwise
};

// Host-side mirror of one axis.
struct AxisHost {
  int M = 1, nspans = 1, p = 0, n = 1, S = 1;
  int pieces = 0;
  int kmode = KMODE_FLOATING;
  int gspans = 1;
  std::vector<int> knots;    // knot positions in span units (t_i = knots[i] / gspans), n + p + 1 of them
  std::vector<double> wts;   // NURBS weights (empty: W = 1)
  std::vector<AxisSub> subs;
  std::vector<int> own_first, own_count, span_start, nL_tab, own_pick;
  std::vector<int2> one_rng;  // per piece: control points owned by it alone, [x, y)
  std::vector<int4> own_tab;
  int bandL_rows = 0, bandU_rows = 0;
};

// Compact launch over operands of very uneven sizes (batches of independent
// fits): block b works on operand op[b], elements base[b] .. base[b] +
// blockDim.x - 1 of it, so the grid holds exactly the tiles that exist.
struct TileMap {
  const int* op = nullptr;
  const long long* base = nullptr;
  int ntiles = 0;
  int threads = 0;  // block size = elements per tile
};

// Streaming multiprocessors of the calling thread's current device (read once
// per device ordinal from cudaDevAttrMultiProcessorCount; 1 if unavailable).
int device_sm_count();

// Dynamic shared-memory limit (and, with `carveout`, the preferred shared
// memory share) of a kernel in the current context, raised to at least
// `bytes` and never lowered, under a process-wide lock (host threads may
// launch the same kernel with different sizes at once).  The attribute
// persists, so a launch that fits the current limit sets nothing.
void ensure_smem_attr(const void* kernel, size_t bytes, bool carveout = false);
template <typename K>
inline void ensure_smem(K kernel, size_t bytes, bool carveout = false) {
  ensure_smem_attr(reinterpret_cast<const void*>(kernel), bytes, carveout);
}

// ---------------------------------------------------------------------------
// kernel launchers (kernels_*.cu)
// ---------------------------------------------------------------------------
void launch_basis(const AxisDev& ax, int* span, double* vd, float* vf, ff* vff, cudaStream_t st);
void launch_gram(const AxisDev& ax, double* AL, cudaStream_t st);
void launch_setup_all(const AxisDev* ax, int naxes, int maxnL, int* status, cudaStream_t st);
void launch_chol(const AxisDev& ax, const double* AL, double* fLd, float* fLf, ff* fLff, double* fUd, float* fUf,
                 ff* fUff, int* status, cudaStream_t st);

template <typename T, typename TIn>
void launch_contract(const LayoutDev& L, int axis, const AxisOp* ops, int nops, int max_out,
                     const TIn* in, T* out, int* status, cudaStream_t st, const TileMap* tm = nullptr);
template <typename T, typename TOut = T>
void launch_expand(const LayoutDev& L, int axis, const AxisOp* ops, int nops, long long max_out,
                   const T* in, TOut* out, cudaStream_t st, const TileMap* tm = nullptr);
template <typename T, typename TQ>
void launch_expand_residual(const LayoutDev& L, int axis, const AxisOp* op, long long nout, const T* in,
                            const TQ* q, double* partials, int nblocks, cudaStream_t st);
template <typename T>
void launch_band_apply(const LayoutDev& L, int axis, const AxisOp* ops, int nops, int max_out,
                       const T* in, T* out, cudaStream_t st);
template <typename T>
void launch_band_solve(const LayoutDev& L, int axis, bool useU, const AxisOp* ops, int nops, int max_fibres,
                       T* x, cudaStream_t st, const TileMap* tm = nullptr);
template <typename T>
void launch_frame_gather(const LayoutDev& L, const long long* offL, int maxL, const T* P, T* Pt, cudaStream_t st);
template <typename T>
void launch_rhs_finalize(const LayoutDev& L, const long long* offL, const long long* offY, int maxU,
                         const T* BL, const T* Y, T* X, cudaStream_t st);
// update rule of the global control points from the owned copies
enum { UPDATE_AVERAGE = 0, UPDATE_OWNER = 1 };
template <typename T>
void launch_average(const LayoutDev& L, const long long* offL, const T* X, T* P, const T* Pprev,
                    unsigned long long* metrics, cudaStream_t st, int rule = UPDATE_AVERAGE);
template <typename T>
void launch_decode_points(const LayoutDev& L, const double* lo, const double* hi, const double* pts, long long npts,
                          const int* deriv, const T* P, void* out, int out_dtype, cudaStream_t st);
template <typename T, typename TQ>
void launch_expand_residual_tiles(const LayoutDev& L, int axis, const AxisOp* ops, const T* in, const TQ* q,
                                  const TileMap& tm, double* tile_part, const int* first, const int* id, int count,
                                  double* out, cudaStream_t st);
void launch_reduce_partials(const double* partials, int nblocks, double* result, cudaStream_t st,
                            double* scratch = nullptr, int scratch_rows = 0);

// Interface jumps (mfa_interface_jumps): one pair of neighbouring subdomains
// along `axis`, left piece index `iface` on that axis.
struct JumpPair {
  int s, t;          // left and right subdomain
  int axis, iface;
  int k0[3], k1[3];  // sample data points [k0, k1) along every axis (one along `axis`)
};
template <typename T>
void launch_interface_jumps(const LayoutDev& L, const long long* offL, const T* X, const T* Pprev, int use_frames,
                            const JumpPair* pairs, int npairs, const double* rows, const int* rowcp, int R,
                            unsigned long long* out, cudaStream_t st);
template <typename TIn, typename TOut>
void launch_cast(const TIn* in, TOut* out, long long n, cudaStream_t st);

// Fused projection: z-planes per staged batch for the largest window, and
// whether cutting every window of the z axis (points k0 .. k0+m-1) into K
// units of whole batches keeps more than P+1 knot spans in every unit.
int proj3d_planes_per_batch(int P, int maxm0, int maxm1, int maxm2, int maxn0, int maxn1);
// First plane of unit b of a window of m2 planes cut into K units of whole
// batches of zb planes (b = K: m2).
int proj3d_unit_start(int m2, int zb, int K, int b);
bool proj3d_split_ok(int P, int zb, int K, long long M, int nspans, long long k0, int m);

template <typename TQ>
bool launch_project3d_ff(const LayoutDev& L, const long long* offL, int maxm0, int maxm1, int maxm2, int maxn0,
                         int maxn1, bool inplace_ok, const TQ* Q, ff* BL, int* status, cudaStream_t st,
                         const AxisOp* inst = nullptr, const int* order = nullptr, int ksplit = 1,
                         ff* zpart = nullptr, unsigned* zctr = nullptr, const int2* units = nullptr,
                         int nunits = 0, bool first = true);

template <typename V, typename TQ, typename TOut, bool RESID>
bool launch_decode3d(const LayoutDev& L, const V* P, const TQ* Q, TOut* out, double* partials, cudaStream_t st);
long long decode3d_tiles(const LayoutDev& L);
bool launch_schwarz3d_ff(const LayoutDev& L, const long long* offL, const int* maxnL, const int* maxnU, const ff* P,
                         const ff* BL, ff* X, cudaStream_t st);
int launch_iter0_3d_ff(const LayoutDev& L, const long long* offL, const int* maxnL, const ff* BL, ff* X,
                       cudaStream_t st);
long long average_ff_blocks(const LayoutDev& L);
void launch_average_ff(const LayoutDev& L, const long long* offL, const ff* X, ff* P, const ff* Pprev, float* part,
                       unsigned long long* metrics, cudaStream_t st, int rule = UPDATE_AVERAGE);

// Batch internals used by the serving runtime (any handle may read a batch).
int batch_decode_points_impl(mfa_handle* h, const mfa_batch* b, int32_t nq, const int32_t* qinst,
                             const int64_t* pt_off, const double* pts, double* out, int on_device);
int batch_instance_ctrl(mfa_handle* h, const mfa_batch* b, int index, double* host_out, int64_t cap);
long long batch_instance_num_ctrl(const mfa_batch* b, int index);

// FP32 data passes of a batch of independent fits (MFA_PREC_FP32): one
// descriptor per instance, pointing into its group's virtual-axis tables.
struct B32Inst {
  int dim, p;
  int M[3], n[3];          // points and control points per axis (1 beyond dim)
  int kbase[3], cbase[3];  // the instance's first point / control point on the group's axes
  long long q_off;         // first data value
  long long x_off;         // first control point in the batch buffer (float-float)
  long long r_off;         // 3-D: first value of its xy-reduced planes (M2 x n1 x n0 floats)
  const int* span[3];      // group tables: first control point of every point
  const float* vals[3];    // FP32 basis values, (p_a + 1) per point
  const int* sstart[3];    // first point of every span number
  int mode;                // 0: a warp stages whole planes (np at a time); 1: up to R rows of one plane
  int np, R;
  int S;                   // x segments per row (at least p knot spans each when S > 1)
};
// One CTA's work: rows [r0, r1) (row = k1 + M1 k2) of one instance, shared by
// nw warps (3-D: by planes; 2-D: by y knot spans, partial sums of the y
// control points at the warps' boundaries in Z from z_off on).
struct B32Item {
  int inst;
  int r0, r1;
  int nw;
  long long z_off;
};
// Shared-memory capacities (elements) of one launch, the maxima over its
// instances: per CTA the x basis values (W per point), the x and y span
// starts, the y basis values (W per row) and the y span of every row; per
// warp the staged rows, the x-reduced rows (and as many y-expanded control
// points for the decode) and the y accumulators of a streamed plane.
struct B32Caps {
  int vb, sx, sy, vy, ysp;
  int stage, xr, ring;
};
constexpr int kB32Threads = 256;
constexpr int kB32ZThreads = 128;  // z contraction: (j1, j0) columns per tile
constexpr int kB32Stage = 1024;  // data values a warp stages per chunk (rows padded to odd pitch)
enum { B32_PROJECT = 0, B32_REFINE = 1, B32_RESIDUAL = 2 };
size_t b32_smem_bytes(const B32Caps& cap, int mode);
// One launch per degree present: items[first[p - 1] .. first[p]) have degree
// p (first has MFA_MAX_DEGREE + 1 entries), with capacities caps[p].
//  B32_PROJECT: N^T q into X (2-D, 1-D) or R (3-D, xy-reduced planes);
//  B32_REFINE: the same for r = q - N P32 (dX in X);
//  B32_RESIDUAL: per item sum of E^2 and max |E|, E = q - N P32, in part.
//  The decode of both takes a 3-D instance's z-expanded control points from
//  DZ (launch_b32_zexpand of the same P32, layout of R).
// With sides (nsides > 0), the launches of successive degrees go to
// sides[(*next_side)++ % nsides] instead of st (the caller forks and joins).
// With only_degree > 0, the launch of that degree alone.
void launch_b32(int mode, const B32Inst* insts, const B32Item* items, const int* first, const B32Caps* caps,
                const float* Q, const float* P32, const float* DZ, ff* X, float* R, float* Z, double* part,
                cudaStream_t st, const cudaStream_t* sides = nullptr, int nsides = 0, int* next_side = nullptr,
                int only_degree = 0);
// P32 = float(X) over tiles of control points (first value, count; at most
// 2^31 values each), after X += dX where dX is not null.
constexpr int kB32CastTile = 4096;
void launch_b32_cast_tiles(const long long* off, const int* len, int ntiles, ff* X, const ff* dX, float* P32,
                           cudaStream_t st);
// DZ (layout of R) = the control points P32 of the tiles' 3-D instances
// expanded along z at every point plane (tiles of 256 values of DZ).
void launch_b32_zexpand(const B32Inst* insts, const int* tile_inst, const long long* tile_base, int ntiles,
                        const float* P32, float* DZ, cudaStream_t st);
void launch_b32_add(ff* X, const ff* dX, long long n, cudaStream_t st);
// z contraction of the xy-reduced planes R of 3-D instances into X (tiles of
// kB32ZThreads (j1, j0) columns of an instance).
void launch_b32_zcontract(const B32Inst* insts, const int* tile_inst, const long long* tile_base, int ntiles,
                          const float* R, ff* X, cudaStream_t st);
void launch_b32_reduce(const int* range, int count, const double* part, double* out, cudaStream_t st);

// One instance of a batch of independent fits, for scattered decode.
struct InstDesc {
  int dim, p;
  int nspans[3], n[3];
  long long cp_off;
};
template <typename T>
void launch_decode_points_inst(const InstDesc* desc, const int* qinst, const long long* pt_off, int nq,
                               long long npts, const double* pts, const T* P, double* out, int p_uniform,
                               cudaStream_t st);  // p_uniform: the degree of every instance, else 0


constexpr int kResidualBlocks = 1216;  // fixed partition of the residual reduction (FP64 partials, any device)
// block sizes of the generic kernels (tile sizes of their TileMaps)
constexpr int kContractThreads = 128, kExpandThreads = 256, kSolveThreads = 64;
// float-float update: at most this many blocks on the shared control points
// (3 per SM of the device, capped; the partials buffer is sized for the cap)
constexpr int kAvgListBlocks = 768;

}  // namespace mfa
