// Instantiation unit of the FFT Helmholtz, state I/O and per-step finish kernels.
#include <algorithm>

#include "dispatch.h"
#include "fft_kernels.cuh"
#include "io_kernels.cuh"
#include "tma.cuh"

namespace apd {

// The timeout path of the bounded waits: thread 0 waits, with the stencil
// kernels' bounded wait and the given limit, on an mbarrier that expects one
// arrival that never comes; when the limit passes it sets the timeout bit of
// the error flags and the kernel returns.  No copy is in flight.
__global__ void k_wait_timeout(unsigned* err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) atomicOr(err, 2u);
}

cudaError_t launch_wait_timeout(unsigned* err, unsigned long long limit_ns, cudaStream_t stream) {
  k_wait_timeout<<<1, 32, 0, stream>>>(err, limit_ns);
  return cudaGetLastError();
}

// The integer-pipe conversions against the instructions, bit for bit (NaN as NaN):
// bad[0] counts mismatching narrowings of the inputs, bad[1] mismatching widenings
// of the narrowed values.
__global__ void k_check_conversions(const double* __restrict__ in, int n, unsigned* __restrict__ bad) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const double d = in[k];
    const float a = narrow_f64_rn(d), b = __double2float_rn(d);
    const bool nb = b != b;
    if (nb ? !(a != a) : __float_as_uint(a) != __float_as_uint(b)) atomicAdd(&bad[0], 1u);
    const double w = widen_f32(b), v = (double)b;
    const bool nv = v != v;
    if (nv ? !(w != w) : __double_as_longlong(w) != __double_as_longlong(v)) atomicAdd(&bad[1], 1u);
  }
}

cudaError_t launch_check_conversions(const double* in, int n, unsigned* bad, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  if (n > 0) k_check_conversions<<<std::min((n + 255) / 256, 4096), 256, 0, stream>>>(in, n, bad);
  return cudaGetLastError();
}
namespace {
template <typename T, int TX, int TY>
MiscSet make_misc() {
  MiscSet m{};
  m.k_finish = reinterpret_cast<const void*>(&k_finish<T, TX, TY>);
  m.k_stage1 = reinterpret_cast<const void*>(&k_stage1<T, TX, TY>);
  m.k_rows_fwd = reinterpret_cast<const void*>(&k_fft_rows_fwd<T>);
  m.k_cols = reinterpret_cast<const void*>(&k_fft_cols<T>);
  m.cols_threads = cols_threads<T>();
  m.rows_threads = rows_threads<T>();
  m.k_rows_inv = reinterpret_cast<const void*>(&k_fft_rows_inv<T>);
  m.k_rows_fwd_bs = reinterpret_cast<const void*>(&k_fft_rows_fwd_bs<T>);
  m.k_cols_bs = reinterpret_cast<const void*>(&k_fft_cols_bs<T>);
  m.k_rows_inv_bs = reinterpret_cast<const void*>(&k_fft_rows_inv_bs<T>);
  m.k_set_state = reinterpret_cast<const void*>(&k_set_state<T>);
  m.k_get_state = reinterpret_cast<const void*>(&k_get_state<T>);
  m.k_diagnostics = reinterpret_cast<const void*>(&k_diagnostics<T>);
  return m;
}
template <typename T>
MiscSet by_tile(int tile) {
  switch (tile) {
    case 0: return make_misc<T, 32, 8>();
    case 1: return make_misc<T, 32, 4>();
    case 2: return make_misc<T, 16, 8>();
    case 3: return make_misc<T, 8, 8>();
    case 4: return make_misc<T, 64, 4>();
    default: return make_misc<T, 32, 16>();
  }
}
}  // namespace

MiscSet misc_set(int f32form, int tile) { return f32form ? by_tile<float>(tile) : by_tile<double>(tile); }
}  // namespace apd
