// Instantiation unit of the FFT Helmholtz, state I/O and per-step finish kernels.
#include "dispatch.h"
#include "fft_kernels.cuh"
#include "io_kernels.cuh"

namespace apd {
namespace {
template <typename T, int TX, int TY>
MiscSet make_misc() {
  MiscSet m{};
  m.k_finish = reinterpret_cast<const void*>(&k_finish<T, TX, TY>);
  m.k_stage1 = reinterpret_cast<const void*>(&k_stage1<T, TX, TY>);
  m.k_rows_fwd = reinterpret_cast<const void*>(&k_fft_rows_fwd<T>);
  m.k_cols = reinterpret_cast<const void*>(&k_fft_cols<T>);
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
