// Host-side waits.
#pragma once

#include <cuda_runtime.h>

namespace rb3 {

// Waits for the stream's work so far with the calling thread asleep, not
// spinning (an event with blocking sync, one per thread): for waits of
// milliseconds on threads that share the host's cores with other waiters.
int wait_stream_blocking(cudaStream_t st);

}  // namespace rb3
