// Guard words around the device arrays (include/mhd.h "guard words"): every
// field of a pool is followed by at least kGuardWords words holding a canary,
// and the pool starts with kGuardWords of them.  They are filled once, when the
// pool is made, and scanned on demand: a canary that changed means some launch
// wrote outside the array it was given.  No kernel of the step reads or writes
// them, so the check costs nothing per step.
#include <climits>
#include <vector>

#include "mhd.h"
#include "mhd_ctx.cuh"
#include "mhd_host.cuh"

namespace mhd {

// A block of guarded fields: [kGuardWords guard][field 0 | guard][field 1 | guard] ...
// with nfields fields of `used` words each, `stride` words apart.
struct GuardBlock {
  double* base;
  int nfields;
  long long stride;
  long long used;
  long long words() const { return kGuardWords + (long long)nfields * (stride - used); }
  // the block offset of guard word i (0 <= i < words())
  __host__ __device__ long long offset(long long i) const {
    if (i < kGuardWords) return i;
    const long long gap = stride - used, j = i - kGuardWords;
    return kGuardWords + (j / gap) * stride + used + j % gap;
  }
};

__global__ void guard_fill_kernel(GuardBlock b, long long n) {
  const double canary = __longlong_as_double((long long)kGuardCanary);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b.base[b.offset(i)] = canary;
}

// The lowest block offset whose word is not the canary, into *first (which the
// caller sets to all ones).
__global__ void guard_scan_kernel(GuardBlock b, long long n, unsigned long long* first) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long o = b.offset(i);
    if ((unsigned long long)__double_as_longlong(b.base[o]) != kGuardCanary) atomicMin(first, (unsigned long long)o);
  }
}

static int guard_grid(long long n) {
  const long long blocks = (n + 255) / 256;
  return (int)(blocks < 1184 ? (blocks < 1 ? 1 : blocks) : 1184);
}

long long guard_stride(long long used) { return (used + 31) / 32 * 32 + kGuardWords; }

long long guard_block_words(int nfields, long long stride) { return kGuardWords + (long long)nfields * stride; }

int guard_fill(cudaStream_t s, double* base, int nfields, long long stride, long long used) {
  GuardBlock b{base, nfields, stride, used};
  const long long n = b.words();
  guard_fill_kernel<<<guard_grid(n), 256, 0, s>>>(b, n);
  CK(cudaGetLastError());
  return MHD_OK;
}

static int guard_scan(cudaStream_t s, const double* base, int nfields, long long stride, long long used,
                      unsigned long long* first_dev) {
  GuardBlock b{const_cast<double*>(base), nfields, stride, used};
  const long long n = b.words();
  guard_scan_kernel<<<guard_grid(n), 256, 0, s>>>(b, n, first_dev);
  CK(cudaGetLastError());
  return MHD_OK;
}

static void guard_decode(unsigned long long off, long long stride, long long used, int* field, long long* word) {
  if (off < (unsigned long long)kGuardWords) {
    *field = 0;
    *word = (long long)off - kGuardWords;  // before field 0: -kGuardWords .. -1
    return;
  }
  const long long j = (long long)off - kGuardWords;
  *field = (int)(j / stride);
  *word = j % stride - used;               // past the field's end: 0, 1, ...
}

int guard_check_blocks(cudaStream_t s, int nblocks, const double* const* bases, const int* nfields,
                       const long long* strides, const long long* used, int* block, int* field, long long* word) {
  *block = -1;
  *field = -1;
  *word = -1;
  if (nblocks <= 0) return MHD_OK;
  unsigned long long* first = nullptr;
  CK(cudaMalloc(&first, sizeof(unsigned long long) * nblocks));
  std::vector<unsigned long long> h(nblocks);
  int rc = MHD_OK;
  if (cudaMemsetAsync(first, 0xff, sizeof(unsigned long long) * nblocks, s) != cudaSuccess) rc = MHD_ERR_CUDA;
  for (int k = 0; k < nblocks && rc == MHD_OK; k++)
    rc = guard_scan(s, bases[k], nfields[k], strides[k], used[k], first + k);
  if (rc == MHD_OK &&
      copy_sync(h.data(), first, sizeof(unsigned long long) * nblocks, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = MHD_ERR_CUDA;
  cudaFree(first);
  if (rc) return rc;
  for (int k = 0; k < nblocks; k++)
    if (h[k] != ULLONG_MAX) {
      *block = k;
      guard_decode(h[k], strides[k], used[k], field, word);
      return MHD_ERR_GUARD;
    }
  return MHD_OK;
}

}  // namespace mhd

using namespace mhd;

int mhd_check_guards(mhd_ctx* c, int* field, long long* word) {
  if (!c || !field || !word) return MHD_ERR_ARG;
  const double* base = c->pool;
  const long long stride = (long long)c->field_elems;
  int block;
  return guard_check_blocks(c->stream, 1, &base, &c->pool_fields, &stride, &c->field_used, &block, field, word);
}

int mhd_guard_layout(const mhd_ctx* c, int* nfields, long long* used, long long* words_after) {
  if (!c || !nfields || !used || !words_after) return MHD_ERR_ARG;
  *nfields = c->pool_fields;
  *used = c->field_used;
  *words_after = (long long)c->field_elems - c->field_used;
  return MHD_OK;
}

int mhd_inject_guard_write(mhd_ctx* c, int field, long long word) {
  if (!c || field < 0 || field >= c->pool_fields) return MHD_ERR_ARG;
  const long long after = (long long)c->field_elems - c->field_used;
  if (word >= after || word < (field == 0 ? -(long long)kGuardWords : 0)) return MHD_ERR_ARG;
  // the word `word` past the field's end (or before field 0's start)
  double* at = c->pool + kGuardWords + (long long)field * (long long)c->field_elems + (word < 0 ? word : c->field_used + word);
  const double zero = 0.0;
  CK(copy_sync(at, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
  return MHD_OK;
}
