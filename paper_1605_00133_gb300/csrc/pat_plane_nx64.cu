// Plane kernels for Nx = 64 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx64(int ny) { return plane_kernels_ny<64>(ny); }
}  // namespace pat
