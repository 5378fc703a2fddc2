// gk_noalloc.cu -- gk_matvec_static: the operator product (A x or A^T x) for
// callers that must not allocate device memory.
//
// Its scratch (control block, f32 copy of x, partial sums of the A^T x kernel)
// lives in g_scratch, a file-scope device array of GK_STATIC_SCRATCH_BYTES that
// every GPU loading this library holds until the process exits.  The host
// never passes the symbol g_scratch itself to a kernel: in host code that name
// is only a stand-in for the device array, so the device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// cached.  A^T x runs the same kernels as gk_matvec; A x runs the row-streaming
// kernel, which needs no partial sums.
#include <mutex>

#include "gk_internal.cuh"

namespace {

constexpr size_t kScratchBytes = GK_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// device address of g_scratch on the current device (set up on first use)
int scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return GK_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return GK_CUDA_ERROR;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GK_OK;
}

// true for device memory of device `dev` (or managed memory): the kernels run on the
// current device and would fault on another GPU's memory without peer access
bool device_pointer(const void *p, int dev) {
  if (p == nullptr) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// true if the byte ranges [a, a + na) and [b, b + nb) share a byte
bool overlap(const void *a, size_t na, const void *b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  return a0 < b0 + nb && b0 < a0 + na;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int gk_matvec_static(const gk_matrix *A, int trans, const double *x, double *y, const gk_opts *opts) {
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return GK_NO_DEVICE;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GK_NO_DEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GK_NO_DEVICE;

  // arguments: the same rules as gk_matvec, and every pointer must be device memory
  if (!A || A->m <= 0 || A->n <= 0 || A->m > INT32_MAX || A->n > INT32_MAX) return GK_INVALID_ARG;
  if (A->dtype < GK_F64 || A->dtype > GK_F16 || !(A->scale == A->scale) || A->scale == 0.0) return GK_INVALID_ARG;
  if (trans != 0 && trans != 1) return GK_INVALID_ARG;
  if (!device_pointer(A->vals, dev) || !device_pointer(x, dev) || !device_pointer(y, dev)) return GK_INVALID_ARG;
  if (A->kind == GK_DENSE) {
    if (A->ld < A->n) return GK_INVALID_ARG;
  } else if (A->kind == GK_CSR) {
    if (!device_pointer(A->rowptr, dev) || !device_pointer(A->colind, dev) || !device_pointer(A->t_vals, dev) ||
        !device_pointer(A->t_rowptr, dev) || !device_pointer(A->t_colind, dev))
      return GK_INVALID_ARG;
  } else {
    return GK_INVALID_ARG;
  }
  // the kernels read x while other blocks write y: the two must not share memory
  if (overlap(x, sizeof(double) * (size_t)(trans ? A->m : A->n), y, sizeof(double) * (size_t)(trans ? A->n : A->m)))
    return GK_INVALID_ARG;

  gk::Op op;
  op.kind = A->kind;
  op.dtype = A->dtype;
  op.m = A->m;
  op.n = A->n;
  op.ld = A->kind == GK_DENSE ? A->ld : 0;
  op.nnz = 0;  // no device read here: CSR products take the default lanes per row
  op.scale = A->scale;
  op.vals = A->vals;
  op.rowptr = A->rowptr;
  op.colind = A->colind;
  op.t_vals = A->t_vals;
  op.t_rowptr = A->t_rowptr;
  op.t_colind = A->t_colind;
  gk::Dev d{sms, dev};

  // scratch layout: [control block][f32 copy of x][partial sums of the A^T x kernel]
  const int64_t nin = trans ? A->m : A->n;
  const size_t ctl_bytes = align256(sizeof(gk::Ctl));
  const size_t x32_bytes = align256(sizeof(float) * (size_t)gk::round_up(A->m > A->n ? A->m : A->n, 64));
  // A^T x keeps one f64 partial sum per (row block, column), the layout k_gemvt_* and
  // k_gemvt_reduce index; the static A x never runs the chunked kernel that needs more
  const int64_t row_blocks = (A->m + gk::gemvt_row_block(op, d) - 1) / gk::gemvt_row_block(op, d);
  const size_t part_bytes = (trans && A->kind == GK_DENSE) ? sizeof(double) * (size_t)row_blocks * (size_t)A->n : 0;
  if (ctl_bytes + x32_bytes + part_bytes > kScratchBytes) return GK_OUT_OF_MEMORY;

  void *base = nullptr;
  const int rc = scratch_address(dev, &base);
  if (rc != GK_OK) return rc;
  gk::Ctl *ctl = reinterpret_cast<gk::Ctl *>(base);
  float *x32 = reinterpret_cast<float *>(static_cast<char *>(base) + ctl_bytes);
  double *part = reinterpret_cast<double *>(static_cast<char *>(base) + ctl_bytes + x32_bytes);

  cudaStream_t s = opts ? (cudaStream_t)opts->stream : nullptr;
  // the array keeps the previous call's contents: the control block (halt flag,
  // arrival counters) must start cleared; x32 and the partial sums are fully
  // overwritten before they are read
  if (gk::reset_ctl(ctl, 0.0, 1, s) != cudaSuccess) return GK_CUDA_ERROR;
  if (gk::copy_vec(nullptr, x32, x, nin, s) != cudaSuccess) return GK_CUDA_ERROR;
  // A x gets no partial-sum buffer: the product then runs the row-streaming kernel,
  // which needs none (the scratch budget above counts partial sums for A^T x only)
  const cudaError_t e = trans ? gk::matvec_t(op, x32, x, y, nullptr, nullptr, part, ctl, s, d)
                              : gk::matvec(op, x32, x, y, nullptr, nullptr, nullptr, ctl, s, d);
  if (e != cudaSuccess) return GK_CUDA_ERROR;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GK_CUDA_ERROR;
  return GK_OK;
}
