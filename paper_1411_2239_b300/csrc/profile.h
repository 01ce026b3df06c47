// Per-kernel CUDA-event instrumentation shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

void rv_prof_begin(const char* name, cudaStream_t s);
void rv_prof_end(cudaStream_t s);
void rv_count_launch();
bool rv_prof_enabled();

#define RV_LAUNCH(name, kernel, grid, block, smem, stream, ...)   \
  do {                                                            \
    rv_prof_begin(name, stream);                                  \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);   \
    rv_prof_end(stream);                                          \
    rv_count_launch();                                            \
  } while (0)
