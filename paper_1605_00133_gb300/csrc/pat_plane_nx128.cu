// Plane kernels for Nx = 128 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx128(int ny) { return plane_kernels_ny<128>(ny); }
}  // namespace pat
