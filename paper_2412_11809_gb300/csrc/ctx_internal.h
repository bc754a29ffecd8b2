// Host-side interface between the contexts (tpc_api.cu) and the serving loop
// (server.cu).  No device code.
#pragma once

#include <cstddef>
#include <mutex>

#include <cuda_runtime.h>

#include "tpc.h"
#include "tpc_internal.cuh"

namespace tpc {

size_t ctx_projected_bytes(tpc_ctx *c, size_t n);   // device bytes once a streaming push of n has run
size_t ctx_held_bytes(tpc_ctx *c);                  // device bytes held now
void ctx_release_scratch(tpc_ctx *c);               // drop work arrays and outputs (idle context)
int ctx_settle(tpc_ctx *c);                         // idle streaming context: learn the exact carry
cudaStream_t ctx_stream(tpc_ctx *c);

// One batched step over contexts with pending hits (their mutexes held by
// the caller), with the lead context's launch choices; consume = false
// leaves the hits pending (a tuning trial).
int batch_step(tpc_ctx **ctxs, int n, bool consume);
int check_batch(tpc_ctx **ctxs, int n);   // the arguments tpc_batch_flush accepts

Tuning &ctx_tuning(tpc_ctx *c);
std::mutex &ctx_mutex(tpc_ctx *c);
size_t ctx_pending(tpc_ctx *c);
void ctx_sensor(tpc_ctx *c, uint32_t *width, uint32_t *height);
int ctx_device(tpc_ctx *c);

}  // namespace tpc
