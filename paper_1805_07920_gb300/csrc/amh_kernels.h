// amh_kernels.h -- launchers of the update kernels (amh_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "amh_device.cuh"

namespace amh {
// random initialisation of every pixel; returns a cudaError_t of the launch
int launch_init(const PhaseArgs& a, cudaStream_t s);
// one colour phase (a.color, a.t); returns a cudaError_t of the launch
int launch_phase(const PhaseArgs& a, cudaStream_t s);
}  // namespace amh
