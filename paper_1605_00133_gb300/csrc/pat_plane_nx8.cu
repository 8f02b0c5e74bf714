// Plane kernels for Nx = 8 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx8(int ny) { return plane_kernels_ny<8>(ny); }
}  // namespace pat
