// Plane kernels for Nx = 256 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx256(int ny) { return plane_kernels_ny<256>(ny); }
}  // namespace pat
