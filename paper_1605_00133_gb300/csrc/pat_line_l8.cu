// Line-pass kernels for lines of length 8 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l8() { return make_line_kernels<8>(); }
}  // namespace pat
