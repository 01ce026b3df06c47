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

// Per-device one-time set-up.  Kernel attributes such as the dynamic
// shared-memory limit apply to the device that is current when they are set,
// so each device of a process needs its own: rv_once_per_device runs fn()
// once per (current device, slot), under a lock; a failed fn() is retried on
// the next call.  rv_num_sms() is the current device's SM count.
constexpr int RV_MAX_DEVICES = 64;
enum { RV_ONCE_FOLD32 = 0, RV_ONCE_FOLD64 = 1, RV_ONCE_FOLD2 = 2, RV_ONCE_BATCH = 3, RV_ONCE_EXTRA = 4,
       RV_ONCE_SLOTS = 8 };
#include "../../include/rv.h"
rv_status rv_once_per_device(int slot, rv_status (*fn)());
int rv_num_sms();
