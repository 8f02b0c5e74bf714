// Plane kernels for Nx = 32 and every supported Ny (one translation unit per Nx, built in parallel).
#include "pat_plane.cuh"

namespace pat {
PlaneKernels plane_kernels_nx32(int ny) { return plane_kernels_ny<32>(ny); }
}  // namespace pat
