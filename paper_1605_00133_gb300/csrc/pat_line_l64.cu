// Line-pass kernels for lines of length 64 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l64() { return make_line_kernels<64>(); }
}  // namespace pat
