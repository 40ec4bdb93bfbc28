// Grid decode that allocates nothing: every intermediate (basis tables and the
// partially expanded arrays between axes) lives in one file-scope static
// device array of fixed size.  Host code only ever uses the array's device
// address obtained with cudaGetSymbolAddress, never the symbol itself.
#include <cuda_runtime.h>

#include "mfa_internal.cuh"

namespace {

// Fixed scratch shared by every call on a device; it stays allocated on every
// GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_decode_scratch[MFA_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the calling thread's current
// context.  Looked up on every call (a table lookup in the runtime that
// queues no stream work), so a context that was torn down and created again,
// where the module may load at another address, never sees a stale pointer.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_decode_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();  // the error came from this lookup
    return MFA_ERR_CUDA;
  }
  *out = static_cast<unsigned char*>(p);
  return MFA_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// One decode stage along `axis`: out has in's shape with n_a control points
// replaced by M_a points; out[k] = sum_r N_{span(k)+r}(u_k) in[span(k)+r].
struct Stage {
  int axis;
  int p;
  long long nin[3];
  long long nout[3];
  const double* in;
  double* out;
  const int* span;
  const double* vals;
};

__global__ void k_expand_static(Stage s) {
  const long long total = s.nout[0] * s.nout[1] * s.nout[2];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const int w = s.p + 1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    long long o[3];
    o[0] = idx % s.nout[0];
    const long long r = idx / s.nout[0];
    o[1] = r % s.nout[1];
    o[2] = r / s.nout[1];
    const long long k = o[s.axis];
    const int j = s.span[k];
    const double* v = s.vals + k * w;
    double acc = 0.0;
    for (int t = 0; t <= s.p; ++t) {
      long long c[3] = {o[0], o[1], o[2]};
      c[s.axis] = j + t;
      acc += v[t] * s.in[c[0] + s.nin[0] * (c[1] + s.nin[1] * c[2])];
    }
    s.out[idx] = acc;
  }
}

}  // namespace

extern "C" int mfa_decode_grid_noalloc(int32_t dim, int32_t degree, const int64_t* npts, const int32_t* nspans,
                                       const double* ctrl, double* out, void* cuda_stream) {
  if (dim < 1 || dim > MFA_MAX_DIM || degree < 1 || degree > MFA_MAX_DEGREE || !npts || !nspans || !ctrl || !out)
    return MFA_ERR_ARG;
  long long M[3] = {1, 1, 1}, n[3] = {1, 1, 1};
  int ns[3] = {1, 1, 1}, p[3] = {0, 0, 0};
  double out_elems = 1.0;
  for (int a = 0; a < dim; ++a) {
    if (npts[a] < 1 || npts[a] > (1LL << 30) || nspans[a] < 1 || nspans[a] > (1 << 30)) return MFA_ERR_ARG;
    M[a] = npts[a];
    ns[a] = nspans[a];
    p[a] = degree;
    n[a] = (long long)nspans[a] + degree;
    out_elems *= (double)M[a];
  }
  if (out_elems > (double)(1LL << 40)) return MFA_ERR_ARG;
  // the intermediate arrays must fit the fixed scratch (checked in floating
  // point first so that huge requests cannot overflow the integer products)
  {
    double cur[3] = {(double)n[0], (double)n[1], (double)n[2]}, need = 0.0;
    for (int a = 0; a < dim - 1; ++a) {
      cur[a] = (double)M[a];
      need += cur[0] * cur[1] * cur[2] * sizeof(double);
    }
    for (int a = 0; a < dim; ++a) need += (double)M[a] * (sizeof(int) + (degree + 1) * 12.0);
    if (need > (double)MFA_NOALLOC_SCRATCH_BYTES) return MFA_ERR_UNSUPPORTED;
  }
  // scratch plan: per axis the span and basis tables (the setup basis kernel
  // also writes an FP32 copy), then the two intermediate stage arrays
  size_t off_span[3], off_vd[3], off_vf[3], used = 0;
  for (int a = 0; a < dim; ++a) {
    off_span[a] = used;
    used = align_up(used + sizeof(int) * (size_t)M[a]);
    off_vd[a] = used;
    used = align_up(used + sizeof(double) * (size_t)M[a] * (degree + 1));
    off_vf[a] = used;
    used = align_up(used + sizeof(float) * (size_t)M[a] * (degree + 1));
  }
  long long stage_elems[2] = {0, 0};
  {
    long long cur[3] = {n[0], n[1], n[2]};
    for (int a = 0; a < dim - 1; ++a) {
      cur[a] = M[a];
      stage_elems[a] = cur[0] * cur[1] * cur[2];
    }
  }
  size_t off_stage[2];
  for (int i = 0; i < 2; ++i) {
    off_stage[i] = used;
    used = align_up(used + sizeof(double) * (size_t)stage_elems[i]);
  }
  if (used > (size_t)MFA_NOALLOC_SCRATCH_BYTES) return MFA_ERR_UNSUPPORTED;

  // a launch error left pending by earlier, unrelated work is not this
  // call's: refuse, and leave it for the code that caused it
  if (cudaPeekAtLastError() != cudaSuccess) return MFA_ERR_CUDA;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MFA_OK) return rc;
  const int grid_cap = 32 * mfa::device_sm_count();
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // basis tables of every axis into the scratch
  const int* span[3] = {nullptr, nullptr, nullptr};
  const double* vals[3] = {nullptr, nullptr, nullptr};
  for (int a = 0; a < dim; ++a) {
    mfa::AxisDev ax{};
    ax.M = (int)M[a];
    ax.nspans = ns[a];
    ax.p = p[a];
    ax.n = (int)n[a];
    int* sp = reinterpret_cast<int*>(base + off_span[a]);
    double* vd = reinterpret_cast<double*>(base + off_vd[a]);
    float* vf = reinterpret_cast<float*>(base + off_vf[a]);
    mfa::launch_basis(ax, sp, vd, vf, nullptr, st);
    if (cudaGetLastError() != cudaSuccess) return MFA_ERR_CUDA;  // this launch failed
    span[a] = sp;
    vals[a] = vd;
  }
  // expand axis 0, then 1, then 2; the last stage writes the caller's output
  const double* in = ctrl;
  long long cur[3] = {n[0], n[1], n[2]};
  for (int a = 0; a < dim; ++a) {
    Stage s{};
    s.axis = a;
    s.p = degree;
    for (int b = 0; b < 3; ++b) s.nin[b] = cur[b];
    cur[a] = M[a];
    for (int b = 0; b < 3; ++b) s.nout[b] = cur[b];
    s.in = in;
    s.out = (a == dim - 1) ? out : reinterpret_cast<double*>(base + off_stage[a]);
    s.span = span[a];
    s.vals = vals[a];
    const long long total = cur[0] * cur[1] * cur[2];
    long long blocks = (total + 255) / 256;
    if (blocks > grid_cap) blocks = grid_cap;
    k_expand_static<<<(unsigned)blocks, 256, 0, st>>>(s);
    if (cudaGetLastError() != cudaSuccess) return MFA_ERR_CUDA;  // this launch failed
    in = s.out;
  }
  return MFA_OK;
}
