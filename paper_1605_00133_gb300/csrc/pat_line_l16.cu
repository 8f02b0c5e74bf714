// Line-pass kernels for lines of length 16 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l16() { return make_line_kernels<16>(); }
}  // namespace pat
