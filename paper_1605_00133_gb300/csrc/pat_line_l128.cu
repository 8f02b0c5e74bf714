// Line-pass kernels for lines of length 128 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l128() { return make_line_kernels<128>(); }
}  // namespace pat
