// amh_kernels.h -- launchers of the update kernels (amh_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "amh_device.cuh"

namespace amh {
// random initialisation of every pixel; returns a cudaError_t of the launch
int launch_init(const PhaseArgs& a, cudaStream_t s);
// one colour phase (a.color, a.t); returns a cudaError_t of the launch
int launch_phase(const PhaseArgs& a, cudaStream_t s);
// One state field (elem bytes per pixel: 16, 4 or 1) between the kernels'
// layout (state_index) and a row-major W x H map in host or device memory.
// Host maps go through a device buffer allocated and freed on the stream.
// Return the first cudaError_t met.
cudaError_t export_state_field(const void* state, void* rows, int W, int H, int elem, bool host, cudaStream_t s);
cudaError_t import_state_field(const void* rows, void* state, int W, int H, int elem, bool host, cudaStream_t s);
}  // namespace amh
