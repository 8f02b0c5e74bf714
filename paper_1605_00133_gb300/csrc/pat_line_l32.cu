// Line-pass kernels for lines of length 32 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l32() { return make_line_kernels<32>(); }
}  // namespace pat
