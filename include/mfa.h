/*
 * mfa.h -- C ABI of the GB300 library for domain-decomposed multivariate
 * functional approximation (MFA): tensor-product B-spline least-squares fits
 * of gridded data, split into overlapping subdomains and made continuous by an
 * overlapping additive-Schwarz iteration.
 *
 * Method: Mahadevan, Lenz, Grindeanu, Peterka, "Parallel Domain Decomposition
 * Techniques Applied to Multivariate Functional Approximation of Discrete
 * Data", arXiv 2210.06528.  Section references below are to that paper.
 *
 * Conventions shared by every call:
 *  - Grids are stored with grid axis 0 fastest in memory: value (i0,i1,i2) of
 *    a grid with npts = (M0,M1,M2) sits at offset i0 + M0*(i1 + M1*i2).
 *    Control points use the same convention with n_a = nspans_a + degree
 *    (more with MFA_KNOTS_CLAMPED, see there).
 *  - Knots on axis a are clamped at the ends and uniform with nspans_a spans
 *    (single interior knots unless MFA_KNOTS_CLAMPED); the data parameters
 *    are u_k = k/(M_a - 1).  Physical coordinates map affinely from
 *    [lo_a, hi_a] to [0, 1].
 *  - Ownership: the caller owns every pointer it passes (q, pts, out, host_out);
 *    the library reads or writes them only inside the call's stream work and
 *    keeps none of them.  Host buffers are copied synchronously with respect
 *    to the host before the call returns; device buffers must stay valid
 *    until the handle's stream has passed the call (mfa_sync).  The library
 *    owns mfa_model and mfa_handle objects until mfa_free / mfa_destroy.
 *  - Errors: argument and layout errors return synchronously with no state
 *    changed.  Errors found on the device (non-positive pivot, non-finite
 *    input) are recorded in a device status word and returned by the next
 *    call that synchronises (mfa_schwarz_iterate, mfa_residual, mfa_get_ctrl,
 *    mfa_sync).  No call traps or aborts the process.
 *  - Threading: a handle and its models are not thread-safe; use one handle
 *    per host thread.  Every call is enqueued on the handle's stream.
 */
#ifndef MFA_GB300_H
#define MFA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfa_handle mfa_handle; /* device, stream, workspace pool */
typedef struct mfa_model mfa_model;   /* a fitted MFA, device resident  */

enum {
  MFA_OK = 0,
  MFA_NOT_CONVERGED = 1,   /* warning: max_iters reached before the tolerance */
  MFA_ERR_ARG = -1,        /* bad pointer, dtype, size or flag */
  MFA_ERR_LAYOUT = -2,     /* layout rejected (core < degree spans, data too sparse, ...) */
  MFA_ERR_OOM = -3,        /* device allocation failed */
  MFA_ERR_CUDA = -4,       /* a CUDA runtime call failed */
  MFA_ERR_NOT_SPD = -5,    /* a local normal matrix had a non-positive Cholesky pivot */
  MFA_ERR_DIVERGED = -6,   /* the Schwarz update grew for 8 iterations in a row */
  MFA_ERR_NONFINITE = -7,  /* the input data held NaN or Inf */
  MFA_ERR_UNSUPPORTED = -8, /* valid request outside what this build implements */
  MFA_ERR_TIMEOUT = -9,     /* a kernel's bounded wait for an asynchronous copy gave up; results invalid */
  MFA_ERR_IO = -10          /* a file could not be read or written, or is not a saved model */
};

enum { MFA_F32 = 0, MFA_F64 = 1 };

/* Arithmetic of the fit.
 * MFA_PREC_FP64 : every step in FP64 (the plain method).
 * MFA_PREC_MIXED: FP64 Gram matrices and Cholesky factors (rounded to FP32
 *                 and float-float copies for the kernels).  Everything else
 *                 runs on the FP32 pipes in float-float arithmetic (a value is
 *                 an unevaluated sum hi + lo of two floats, about 48 bits):
 *                 basis values, the projection N^T Q, the iteration-0 solves,
 *                 the Schwarz residual B_U - A_{U,L} Z, the averaging and its
 *                 metrics, decode and residual.  The correction solve of each
 *                 Schwarz step is plain FP32 (iterative refinement: its
 *                 right-hand side is the float-float residual, so it adds no
 *                 rounding floor at the fixed point).  Residual reductions
 *                 sum E^2 in float-float and widen only per-tile totals to
 *                 FP64.  FP64 input data are carried exactly (as float-float)
 *                 through the projection and the residual.
 *                 Accuracy: decoded RMS within 1 % of the FP64 fit's and
 *                 control points within about 1e-9 relative of it.
 * MFA_PREC_FP32 : (batches of independent fits and the server) FP32 basis
 *                 values, FP32 projection N^T Q and FP32 decode / residual,
 *                 read straight from FP32 data; FP64 Gram matrices and
 *                 Cholesky factors; banded solves in float-float (about 48
 *                 bits) with the factors' float-float copies; control points
 *                 kept as float-float and read back as FP64.  An instance
 *                 whose a-priori FP32 error bound 2^-24 prod_a
 *                 sqrt(cond(N_a^T N_a)) exceeds 2e-6 of the data range gets
 *                 one step of iterative refinement (r = q - N P decoded and
 *                 projected in FP32 from the FP32 copy of P, solved, added).
 *                 For fits whose error is far above FP32 rounding of the data
 *                 (a decoded RMS of at least 100 x 2^-24 x the data range
 *                 keeps the FP32 error below 1 % of the RMS); FP32 data only,
 *                 and MFA_ERR_UNSUPPORTED for an instance outside the
 *                 kernels' staging limits (points along axis 0 <= 1023,
 *                 control points along axis 0 <= 256, W x points along axis 0
 *                 <= 8192 with W = 4 for degree <= 3 and 8 above). */
enum { MFA_PREC_FP64 = 0, MFA_PREC_MIXED = 1, MFA_PREC_FP32 = 2 };

#define MFA_MAX_DIM 3
#define MFA_MAX_DEGREE 7

/* Knots at the subdomain interfaces (Sec. 2.2; Sec. 3.1.1 "Comparison of
 * Clamped vs Floating Boundary Knots").
 * MFA_KNOTS_FLOATING: single interior knots; neighbours share the p control
 *                     points straddling an interface and the converged fit
 *                     is C^{p-1} there (the paper's method).
 * MFA_KNOTS_CLAMPED : every interface breakpoint is repeated p times, so each
 *                     core carries its own clamped uniform knot vector and
 *                     neighbours share exactly one control point, the value at
 *                     the interface; the fit is C^0 there and depends on the
 *                     subdomain count.  Axis a then has
 *                     n_a = nspans[a] + degree + (degree - 1)(nsub[a] - 1)
 *                     control points. */
enum { MFA_KNOTS_FLOATING = 0, MFA_KNOTS_CLAMPED = 1 };

/* Problem layout (Sec. 2.2, Eq. vecp-layout; Algorithm 1 parameters N, p).
 *   dim          1..3
 *   degree       p, 1..MFA_MAX_DEGREE, same on every axis
 *   npts[a]      data points M_a on axis a (>= 1; axes >= dim are ignored)
 *   nspans[a]    global knot spans; n_a = nspans[a] + degree control points
 *   nsub[a]      subdomains along axis a (N = product)
 *   core_spans[a] NULL for an even split (the first nspans % nsub cores get
 *                one span more) or an array of nsub[a] span counts summing to
 *                nspans[a]; with nsub[a] > 1 every core needs >= degree spans
 *   overlap[a]   delta, extra knot spans shared per interior side (Sec. 2.2,
 *                "Augmenting Knot Spans with Overlap"), >= 0
 *   precision    MFA_PREC_FP64 or MFA_PREC_MIXED
 *   lo[a], hi[a] physical extent of axis a (used by scattered decode)
 *   knots        MFA_KNOTS_FLOATING (the default, 0) or MFA_KNOTS_CLAMPED
 *   weights[a]   NULL (B-splines, W = 1) or n_a positive control-point
 *                weights of axis a (host memory, read during mfa_encode): the
 *                NURBS basis of Sec. 2.1, Eq. nurbs-basis, with the separable
 *                weights W_g = W_0[g_0] W_1[g_1] W_2[g_2], so the rational
 *                basis is a tensor product and the fit stays separable.  The
 *                weights are fixed, so the Schwarz update of the weighted
 *                control points P W (Sec. 4) equals the update of P. */
typedef struct {
  int32_t dim;
  int32_t degree;
  int64_t npts[3];
  int32_t nspans[3];
  int32_t nsub[3];
  const int32_t* core_spans[3];
  int32_t overlap[3];
  int32_t precision;
  double lo[3];
  double hi[3];
  int32_t knots;
  const double* weights[3];
} mfa_layout;

/* Convergence and error metrics (Algorithm 1: "update local error",
 * "check convergence metrics").
 *   iters        Schwarz iterations done on this model (0 right after encode)
 *   dP_rel       max|P^k - P^{k-1}| / max|P^k| of the last iteration
 *   jump_max     largest spread (max - min) among the owned copies of any
 *                shared control point: the jump residual F_ij of
 *                Eq. (nonlinear-residuals) measured in control-point space
 *   rms_decoded, maxabs_decoded   RMS and max |Q - R P| over all data
 *   data_range   max(Q) - min(Q)
 *   jump_orders  number of entries of jump_deriv filled by
 *                mfa_interface_jumps (0 otherwise)
 *   jump_deriv[r] largest jump of the r-th derivative across any subdomain
 *                interface between the local splines of the two neighbours
 *                (Sec. 2.2: C^0 .. C^{p-1}; see mfa_interface_jumps)       */
typedef struct {
  int32_t iters;
  int32_t status;
  double dP_rel;
  double jump_max;
  double rms_decoded;
  double maxabs_decoded;
  double data_range;
  int32_t jump_orders;
  int32_t pad_;
  double jump_deriv[MFA_MAX_DEGREE + 1];
} mfa_report;

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  The handle owns a
 * stream-ordered memory pool for models and scratch.  Returns MFA_OK. */
int mfa_create(int device, void* cuda_stream, mfa_handle** out);

/* Release the handle and its pool.  Models must be freed first. */
int mfa_destroy(mfa_handle* h);

/* Setup and iteration 0 of Algorithm 1 (Sec. 2.4): build the subdomain
 * layout, evaluate the Cox-de Boor basis of every axis (Sec. 2.1, Eq.
 * nurbs-basis, W = 1), assemble and Cholesky-factor the banded per-axis
 * normal matrices of every subdomain window (Sec. 2.3.1), project the window
 * data onto every subdomain's control points (N^T Q), solve the decoupled
 * unconstrained local LSQ problems (Eq. minimization-problem) and average the
 * owned copies with weight 1/n_s (Sec. 2.3.2) into the global iterate P^0.
 *   q            grid of prod(npts) values, dtype q_dtype (MFA_F32/MFA_F64),
 *                on the device if q_on_device, else in host memory
 *   out          receives a new model (free with mfa_free)
 * Asynchronous on the handle's stream except for host input copies. */
int mfa_encode(mfa_handle* h, const mfa_layout* layout, const void* q, int q_dtype,
               int q_on_device, mfa_model** out);

/* Outer iterations k >= 1 of Algorithm 1 (Sec. 2.3.2): exchange the frame
 * control points of every subdomain from the lagged global iterate (a device
 * gather), re-solve every subdomain with its frame held fixed (the Schur
 * decoupling of Eq. global-system, done in control-point space without
 * re-reading the data), and average the owned copies into P^k.
 * Stops ("check convergence metrics") after the first iteration k with
 *   dP_rel <= tol_dP                                (tol_dP > 0), or
 *   |RMS_k - RMS_{k-1}| <= tol_rms_stall * RMS_k     (tol_rms_stall > 0),
 * where RMS_k is the decoded RMS error of P^k over all data (RMS_0 that of
 * the encode's P^0), or after max_iters iterations.  The stall test decodes
 * the full grid once per iteration against the data given to mfa_encode:
 * host data were staged there; device data must still be valid and
 * unchanged.  Returns MFA_OK when a tolerance was met, MFA_NOT_CONVERGED
 * when max_iters ran out (both tolerances <= 0 always run max_iters), or an
 * error.  `rep` (may be NULL) receives iters, dP_rel, jump_max and, with the
 * stall test, rms_decoded, maxabs_decoded and data_range of the last
 * iterate. */
int mfa_schwarz_iterate(mfa_handle* h, mfa_model* m, int32_t max_iters, double tol_dP,
                        double tol_rms_stall, mfa_report* rep);

/* Continuity across subdomain interfaces (Sec. 2.2: C^0 .. C^{p-1};
 * Algorithm 1 "check convergence metrics").  For every pair of subdomains
 * that are neighbours along an axis a, their local splines -- the control
 * points each used in its last solve: its owned copy plus the frame values
 * it held (after mfa_encode: its whole unconstrained local solution) -- are
 * evaluated at the interface breakpoint, the left one as a left limit and the
 * right one as a right limit, at every data point of the pair's common core
 * along the other axes.  jump r is the largest |difference| of the r-th
 * derivative along a, taken with respect to the knot coordinate
 * x = u * nspans[a] (so every order has the scale of the data), over all
 * pairs and samples.  Fills rep->jump_deriv[0..max_order] and
 * rep->jump_orders = max_order + 1 (0 <= max_order <= degree); with overlap
 * >= degree a converged floating-knot fit has jumps at rounding level for
 * r < p.  A model with one subdomain has no interfaces and reports zeros.
 * Synchronous; computed in FP64 from the model's values. */
int mfa_interface_jumps(mfa_handle* h, const mfa_model* m, int32_t max_order, mfa_report* rep);

/* Decode the global MFA (Algorithm 1 error step, R P; Sec. 2.1 derivatives).
 *   pts == NULL  full data grid: writes prod(npts) values in grid layout
 *   pts != NULL  npts_q scattered points, row-major [npts_q][dim] physical
 *                coordinates (clamped to [lo, hi])
 *   deriv        NULL for values, else per-axis derivative orders (each
 *                0..degree) of the mixed partial derivative with respect to
 *                the physical coordinates
 *   out          dtype out_dtype, on the device if out_on_device            */
int mfa_decode(mfa_handle* h, const mfa_model* m, const double* pts, int64_t npts_q,
               const int32_t* deriv, void* out, int out_dtype, int out_on_device);

/* Persistence of a fitted model (the paper writes the encoded MFA to disk
 * for later decoding, Algorithm 1 output).  mfa_save writes the layout, the
 * update rule, the iteration count and the global control points exactly as
 * held on the device (FP64, or float-float pairs for MFA_PREC_MIXED), plus,
 * with flags & MFA_SAVE_STATE, the Schwarz state (B_L and the subdomain
 * copies) so the iteration can continue after a load.  mfa_load rebuilds the
 * model on the handle's device (layout, basis, factors) and restores those
 * values bit for bit; a model loaded without state decodes and computes
 * residuals but mfa_schwarz_iterate refuses it (MFA_ERR_ARG).  Files are
 * little-endian and carry a magic and a version; anything else is refused
 * with MFA_ERR_IO.  Not for batch models.  Synchronous. */
#define MFA_SAVE_STATE 1
int mfa_save(mfa_handle* h, const mfa_model* m, const char* path, int flags);
int mfa_load(mfa_handle* h, const char* path, mfa_model** out);

/* Update rule of the global control points from the subdomains' owned
 * copies (Sec. 2.3).  MFA_UPDATE_AVERAGE (the default): the uniformly
 * weighted average, w = 1/n_s.  MFA_UPDATE_OWNER: every control point takes
 * the copy of the subdomain whose core holds its Greville abscissa
 * (t_{g+1} + ... + t_{g+p})/p, per axis (restricted additive Schwarz); with
 * overlap >= degree both rules have the global fit as their fixed point.
 * Setting the rule recomputes the current global control points from the
 * copies the model holds (after mfa_encode: the iteration-0 copies), so the
 * rule applies to every update that follows.  Not for batch models. */
enum { MFA_UPDATE_AVERAGE = 0, MFA_UPDATE_OWNER = 1 };
int mfa_set_update_rule(mfa_handle* h, mfa_model* m, int rule);

/* The per-subdomain comparator form of encode + Schwarz iteration (the
 * plain FP64 method as a straightforward GPU port would run it; no
 * counterpart entry point in the paper, which runs one MPI task per
 * subdomain): the same arithmetic as MFA_PREC_FP64, but every data-sized
 * stage (projection of the window data, band products, banded solves) is one
 * launch per subdomain and axis, and every Schwarz iteration re-reads the
 * window data from q to rebuild the local right-hand sides.  Requires
 * lay->precision == MFA_PREC_FP64.  Device data must stay valid until the
 * call returns (it synchronises); host data are staged once.  Runs up to
 * max_iters iterations (stop at dP_rel <= tol_dP) and returns the fitted
 * model, usable with every other call, in *out; statuses as
 * mfa_schwarz_iterate (on a negative status no model is returned). */
int mfa_encode_plain(mfa_handle* h, const mfa_layout* lay, const void* q, int q_dtype, int q_on_device,
                     int32_t max_iters, double tol_dP, mfa_report* rep, mfa_model** out);

/* Decoded error E = Q - R P over the full grid (Algorithm 1 "update local
 * error"): fills rep->rms_decoded, maxabs_decoded, data_range.  Synchronous.
 * q == NULL uses the device copy that mfa_encode made of host data for this
 * model (kept until mfa_free), so a host-data encode plus its residual moves
 * the data across the link once; MFA_ERR_ARG if the model was encoded from
 * device data (q_dtype and q_on_device are then ignored). */
int mfa_residual(mfa_handle* h, const mfa_model* m, const void* q, int q_dtype,
                 int q_on_device, mfa_report* rep);

/* Copy the global control points (FP64, grid layout, prod(n_a) values) to
 * host memory; cap is the capacity of host_out in values.  Synchronous. */
int mfa_get_ctrl(mfa_handle* h, const mfa_model* m, double* host_out, int64_t cap);

/* The same copy, enqueued: the FP64 cast runs on the handle's stream and the
 * copy to host_out on the handle's copy stream, so later calls (mfa_residual,
 * another encode) proceed beside it.  host_out must stay valid, and holds the
 * values only once mfa_sync(h) has returned; pinned memory keeps the copy
 * asynchronous.  Errors as mfa_get_ctrl; copy errors surface at mfa_sync. */
int mfa_get_ctrl_async(mfa_handle* h, const mfa_model* m, double* host_out, int64_t cap);

/* Number of global control points of a model (prod n_a), or < 0 on error. */
int64_t mfa_num_ctrl(const mfa_model* m);

/* Free a model (stream-ordered on the stream of the handle that made it). */
int mfa_free(mfa_model* m);

/* Wait for the handle's stream and its copy stream (asynchronous reads);
 * return and clear the device status word. */
int mfa_sync(mfa_handle* h);

/* Static text for a status code. */
const char* mfa_status_string(int status);

/* The layout of one axis, built on the host exactly as mfa_encode builds it
 * (Sec. 2.2: subdomain cores, the overlap delta in knot spans, the data each
 * subdomain fits, its local control points, and the owner of every control
 * point for the owner-takes update of Sec. 2.3).  No device is touched, so
 * this runs on a machine without a GPU.
 *   npts, nspans, degree   grid points, global knot spans and p of the axis
 *   nsub, core_spans       subdomains and their core spans (NULL: even
 *                          split, the extra spans to the first subdomains)
 *   overlap                delta, in knot spans
 *   knots                  MFA_KNOTS_FLOATING or MFA_KNOTS_CLAMPED
 *   out                    caller-owned, cap >= nsub rows of 10 int32 values,
 *                          row s = { a, b, w0, w1, k0, k1, l0, nL, oU, nU }:
 *                          core spans [a, b); window spans [w0, w1) (the core
 *                          widened by delta, clipped); data points k0..k1
 *                          (parameters k/(npts-1) in the closed window
 *                          interval); local control points l0 .. l0+nL-1, of
 *                          which l0+oU .. l0+oU+nU-1 are owned
 *   owner                  caller-owned, n int32 values (n = nspans + degree,
 *                          plus (degree - 1)(nsub - 1) for clamped knots) or
 *                          NULL: the subdomain whose core holds control point
 *                          g's Greville abscissa
 * Returns MFA_OK; MFA_ERR_ARG for sizes out of range or cap < nsub;
 * MFA_ERR_LAYOUT for this axis's rejections in mfa_encode (a core of fewer
 * than degree spans between interfaces, or a window whose collocation matrix
 * fails the Schoenberg-Whitney condition).  Nothing is written on an error. */
int mfa_axis_layout(int64_t npts, int32_t nspans, int32_t degree, int32_t nsub, const int32_t* core_spans,
                    int32_t overlap, int32_t knots, int32_t* out, int32_t cap, int32_t* owner);

/* Condition number of one axis's normal matrix N^T N (Sec. 2.3.1), as the
 * FP32 data passes estimate it on the host: npts points u_k = k / (npts - 1),
 * a clamped uniform knot vector of nspans spans, B-spline basis of the given
 * degree (Sec. 2.1).  An MFA_PREC_FP32 batch gives an instance one
 * refinement step when 2^-24 times the product over its axes of the square
 * root of this value exceeds 2e-6.  The estimate: the banded matrix in FP64,
 * 30 power iterations for its largest eigenvalue and 30 inverse iterations
 * (banded Cholesky solves) for its smallest.  Host only; no GPU is used.
 *   *out  the estimate; 1e300 where N^T N is not positive definite (a span
 *         without enough points)
 * Returns MFA_OK; MFA_ERR_ARG for npts < 1, nspans < 1, a degree outside
 * 1..MFA_MAX_DEGREE or a NULL out (nothing written). */
int mfa_gram_condition(int64_t npts, int32_t nspans, int32_t degree, double* out);

/* Grid decode that allocates nothing.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory at the point where they decode: for example
 * an analysis or visualisation plugin running inside a simulation that has
 * already reserved the whole device through its own memory pool (so a new
 * allocation would fail or break the host application's budget), or a loop
 * that must not stall because cudaMalloc / cudaFree may synchronise the
 * device.  Such a caller passes its own input and output buffers and the
 * call uses no other memory than one fixed scratch array.
 *
 * Decodes the tensor-product B-spline with clamped uniform knots (nspans[a]
 * spans, degree `degree`) on its full data grid u_k = k/(npts[a]-1), the same
 * values as mfa_decode with pts == NULL.
 *   dim, degree, npts[dim], nspans[dim]  as in mfa_layout
 *   ctrl    device pointer, prod(nspans[a] + degree) FP64 control points,
 *           grid layout (axis 0 fastest)
 *   out     device pointer, prod(npts[a]) FP64 values, grid layout
 *   cuda_stream  stream of the current device on which the work is queued
 * Runs on the calling thread's current device, which must own ctrl, out and
 * the stream.  Asynchronous; the caller owns ctrl and out.
 *
 * Memory: basis tables and the intermediate arrays between axes live in one
 * static device array of MFA_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into the
 * library; every GPU that loads the library holds it until the process
 * exits.  The call never calls cudaMalloc, cudaFree or any allocating
 * routine.  A request whose basis tables and intermediates exceed the array
 * returns MFA_ERR_UNSUPPORTED before any work is queued (roughly: 2-D grids
 * up to npts[0] * (nspans[1] + degree) of 4M values, 3-D grids whose
 * npts[0]*npts[1]*(nspans[2]+degree) stays near 3M values).
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which queues no stream work), so the address stays
 * right after the context is torn down and created again.  The first call
 * on a device also loads the library's device code there: make that first
 * call before any stream capture.  All calls on a device share the array and
 * it keeps the last call's contents (every element a call reads was written
 * by that call first, so nothing needs clearing); calls whose GPU work
 * overlaps in time, on different streams or from different host threads,
 * race on the array and must be serialised by the caller.
 * Returns MFA_OK, MFA_ERR_ARG, MFA_ERR_UNSUPPORTED or MFA_ERR_CUDA.
 * MFA_ERR_CUDA is returned without queueing anything when a launch error
 * from earlier work is still pending on the calling thread (that error is
 * left in place for its owner), and after a launch of this call fails. */
#define MFA_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int mfa_decode_grid_noalloc(int32_t dim, int32_t degree, const int64_t* npts, const int32_t* nspans,
                            const double* ctrl, double* out, void* cuda_stream);

/* ---- Batches of independent fits -----------------------------------------
 * Many separate grids, each fitted on its own (one subdomain, N = 1: the
 * global LSQ of Eq. minimization-problem), in a handful of launches for the
 * whole batch instead of a set of launches per grid.  The paper fits one
 * field at a time; the batch form serves workloads of thousands of small
 * uneven fits.  Instances may differ in dimension, degree, grid and knot
 * spans; they are grouped by (dimension, degree) and every group runs the
 * projection, banded solves and decode as single launches over all of its
 * instances.
 *
 * Data: one array of q_dtype values; instance i's grid (axis 0 fastest, the
 * same convention as a single fit) starts at inst[i].q_offset.  Knots per
 * axis are clamped uniform with nspans spans (nspans + degree control
 * points) and u_k = k/(M-1), as for a single fit.  precision is
 * MFA_PREC_FP64, MFA_PREC_MIXED (float-float data passes, FP64
 * factorisation) or MFA_PREC_FP32 (FP32 data passes, FP64 solves).  Host data are staged once (kept for the residual with
 * q == NULL); device data must stay valid until the call returns.
 * Layout errors (Schoenberg-Whitney precheck per instance) return
 * MFA_ERR_LAYOUT with no batch created. */
typedef struct {
  int32_t dim;        /* 1..MFA_MAX_DIM */
  int32_t degree;     /* 1..MFA_MAX_DEGREE */
  int64_t npts[3];    /* grid points per axis (entries beyond dim ignored) */
  int32_t nspans[3];  /* knot spans per axis (entries beyond dim ignored) */
  int64_t q_offset;   /* index of the instance's first value in the data array */
} mfa_instance;

typedef struct mfa_batch mfa_batch;

int mfa_encode_batch(mfa_handle* h, int32_t count, const mfa_instance* inst, const void* q, int q_dtype,
                     int q_on_device, int precision, mfa_batch** out);

/* Refit the batch's instances to new data with the same layout (same
 * instances and offsets): the projection and solves of every group run as
 * one captured CUDA graph (captured on the first refit, replayed after).
 * q must be device data, valid until the call returns; synchronous. */
int mfa_batch_refit(mfa_handle* h, mfa_batch* b, const void* q, int q_dtype);

/* Block sizes of the batch's launches (sizes[0] projection, [1] banded
 * solves, [2] decode) of its first group.  The first mfa_batch_refit tunes
 * every (dimension, degree) group on its own (mfa_batch_group_tuning);
 * candidate_ms (9 floats, may be NULL) gets, for FP64 and mixed batches, the
 * sum over the groups of each tiled candidate's fit time, row-major by
 * projection size (64/128/256 threads) x solve size (32/64/128).  Returns
 * MFA_OK once tuned, MFA_NOT_CONVERGED before the first refit (defaults
 * 128/64/256). */
int mfa_batch_tile_sizes(const mfa_batch* b, int32_t* sizes, float* candidate_ms);

/* Tuning of one (dimension, degree) group of a batch (group 0 ..
 * mfa_batch_info().groups - 1), chosen by timing on the first refit.  The
 * paper has no counterpart (a report of this library's autotuner).
 *   FP64 / mixed batches: candidate_ms[3 i + j] = the group's fit with
 *     projection blocks of 64/128/256 (i) and solve blocks of 32/64/128 (j)
 *     threads; candidate_ms[9] = its fused one-CTA-per-instance 3-D path
 *     (mixed 3-D groups; -1 otherwise); the fastest is kept (`fused`,
 *     tile_c, tile_s).  The fused path sums in another order than the tiled
 *     one, so the choice can change the fit's last bits (both within the
 *     FP64 bar); block sizes never do.
 *   FP32 batches: candidate_ms[0..2] = the group's solves with 32/64/128
 *     threads; candidate_ms[3..5] = the batch's FP32 projection with CTA
 *     items of about 16 K / 32 K / 128 K points (`item_pts` is the
 *     batch-wide choice; neither changes the fit).
 * chosen_ms is the kept candidate's time.  Returns MFA_NOT_CONVERGED before
 * the first refit. */
#define MFA_TUNE_CANDIDATES 10
typedef struct mfa_group_tuning_t {
  int32_t dim, degree, instances;
  int32_t tile_c, tile_s, tile_e;
  int32_t fused;
  int32_t item_pts;
  float chosen_ms;
  float candidate_ms[MFA_TUNE_CANDIDATES];
} mfa_group_tuning_t;
int mfa_batch_group_tuning(const mfa_batch* b, int32_t group, mfa_group_tuning_t* out);

/* Shape of a batch: instances, (dimension, degree) groups, precision, and
 * for MFA_PREC_FP32 the instances that get a refinement step and the CTA
 * items of the data passes; data points and control points in total.  The
 * paper has no counterpart (a report of this library's batching). */
typedef struct mfa_batch_info_t {
  int32_t count;
  int32_t groups;
  int32_t precision;
  int32_t refined;
  int32_t items;
  int32_t reserved;
  int64_t points;
  int64_t ctrl;
} mfa_batch_info_t;
int mfa_batch_info(const mfa_batch* b, mfa_batch_info_t* out);

/* Control points of every instance, concatenated in instance order (each
 * instance in its own grid layout, axis 0 fastest, prod(nspans_a + degree)
 * values).  mfa_batch_ctrl_offsets writes count + 1 offsets into it.
 * mfa_batch_get_ctrl copies FP64 values to host memory (cap = capacity in
 * values); synchronous. */
int64_t mfa_batch_num_ctrl(const mfa_batch* b);
int mfa_batch_ctrl_offsets(const mfa_batch* b, int64_t* host_off);
int mfa_batch_get_ctrl(mfa_handle* h, const mfa_batch* b, double* host_out, int64_t cap);

/* Decoded error of every instance against its data (q == NULL: the copy
 * staged from host data): rms[i] and maxabs[i] (host arrays of count
 * doubles).  Synchronous. */
int mfa_batch_residual(mfa_handle* h, const mfa_batch* b, const void* q, int q_dtype, int q_on_device,
                       double* rms, double* maxabs);

/* Decode every instance on its own grid into out (out_dtype values laid out
 * like the data: instance i at inst[i].q_offset). */
int mfa_batch_decode(mfa_handle* h, const mfa_batch* b, void* out, int out_dtype, int out_on_device);

/* Scattered decode of batch instances: query k evaluates instance qinst[k]
 * at the points pts[pt_off[k] .. pt_off[k+1]), three doubles per point (the
 * parameters u in [0,1] along axes 0, 1, 2, clamped; entries beyond the
 * instance's dimension are ignored), writing one FP64 value per point into
 * out.  All arrays on the host (on_device = 0) or all on the device; nq >= 1,
 * offsets non-decreasing from pt_off[0] = 0.  Synchronous. */
int mfa_batch_decode_points(mfa_handle* h, const mfa_batch* b, int32_t nq, const int32_t* qinst,
                            const int64_t* pt_off, const double* pts, double* out, int on_device);

int mfa_batch_free(mfa_batch* b);

/* ---- Serving: continuous batching of encode requests and decode queries --
 * No counterpart in the paper (which encodes one field per run); this is the
 * serving form of the batch of independent fits.  Requests arrive from any
 * host thread and get an id (> 0; a negative value is an error status).
 * Admission is first come, first served against mem_budget bytes of device
 * memory: an encode reserves its staged data, scratch and resident model, a
 * decode its points and values; a request that alone exceeds the budget is
 * refused with MFA_ERR_OOM.  `workers` threads each own a handle and a CUDA
 * stream; a free worker takes every admitted request of one kind (encodes of
 * one precision, at most max_batch of them, or decodes of resident models)
 * as one job, so jobs overlap on the device and requests arriving meanwhile
 * join the next job.
 *   mfa_server_encode  fit one grid (FP32 data on the host, layout as one
 *                      mfa_instance, q_offset ignored); the id names the
 *                      model, which stays resident until mfa_server_release
 *   mfa_server_decode  evaluate a model at npts points (3 doubles each: the
 *                      parameters u in [0,1] per axis) into out (npts doubles);
 *                      may be submitted while the model is still being fitted
 *   mfa_server_wait    block until a request is done (timeout_s <= 0: no
 *                      limit; MFA_ERR_TIMEOUT when it ran out), returning its
 *                      status and timestamps (seconds since the server was
 *                      created)
 * The caller's buffers (data, points, values) must stay valid until the
 * request is done.  mfa_server_destroy releases every model and joins the
 * workers after the queued work. */
typedef struct mfa_server mfa_server;
typedef struct {
  int32_t status;  /* MFA_OK or an error status */
  int32_t kind;    /* 0 encode, 1 decode */
  double t_submit, t_admit, t_start, t_done;
} mfa_request_info;
typedef struct {
  int64_t budget, reserved, peak_reserved; /* bytes */
  int64_t queued, resident_models, encode_jobs, decode_jobs;
} mfa_server_stats_t;

int mfa_server_create(int device, int32_t workers, int64_t mem_budget, int32_t max_batch, mfa_server** out);
int64_t mfa_server_encode(mfa_server* s, const mfa_instance* inst, const void* host_q, int precision);
int64_t mfa_server_decode(mfa_server* s, int64_t model, int64_t npts, const double* host_pts, double* host_out);
int mfa_server_wait(mfa_server* s, int64_t id, double timeout_s, mfa_request_info* info);
int mfa_server_release(mfa_server* s, int64_t model);
int64_t mfa_server_num_ctrl(mfa_server* s, int64_t model);
int mfa_server_get_ctrl(mfa_server* s, int64_t model, double* host_out, int64_t cap);
int mfa_server_stats(mfa_server* s, mfa_server_stats_t* st);
int mfa_server_destroy(mfa_server* s);

/* Tracing (per-phase timing of Algorithm 1's steps, as in the paper's
 * setup / solve / iterate / decode breakdown, Sec. 3.2.4).  When enabled,
 * every kernel launch of the handle is bracketed by CUDA events on the
 * handle's stream and its duration is added to its kernel class.  Launch
 * counts are kept whether or not timing is enabled.
 *   mfa_trace_enable  enable (1) / disable (0) event timing; resets totals
 *   mfa_trace_read    synchronises the stream, then returns the total
 *                     milliseconds and launch count of kernel class `cls`
 *                     since the last reset (cls in 0..MFA_TRACE_CLASSES-1)
 *   mfa_trace_name    static name of a kernel class                        */
#define MFA_TRACE_CLASSES 16
int mfa_trace_enable(mfa_handle* h, int enable);
int mfa_trace_read(mfa_handle* h, int32_t cls, double* total_ms, int64_t* launches);
const char* mfa_trace_name(int32_t cls);

#ifdef __cplusplus
}
#endif

#endif /* MFA_GB300_H */
