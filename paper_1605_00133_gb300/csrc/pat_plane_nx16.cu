// Plane kernels for Nx = 16 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx16(int ny) { return plane_kernels_ny<16>(ny); }
}  // namespace pat
