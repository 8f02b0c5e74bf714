// Line-pass kernels for lines of length 256 (one translation unit per length, compiled in parallel).
#include "pat_line.cuh"

namespace pat {
LineKernels line_kernels_l256() { return make_line_kernels<256>(); }
}  // namespace pat
