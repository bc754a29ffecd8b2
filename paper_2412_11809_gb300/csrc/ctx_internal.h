// Host-side interface between the contexts (tpc_api.cu) and the serving loop
// (server.cu).  No device code.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "tpc.h"

namespace tpc {

size_t ctx_projected_bytes(tpc_ctx *c, size_t n);   // device bytes once a streaming push of n has run
size_t ctx_held_bytes(tpc_ctx *c);                  // device bytes held now
void ctx_release_scratch(tpc_ctx *c);               // drop work arrays and outputs (idle context)
int ctx_settle(tpc_ctx *c);                         // idle streaming context: learn the exact carry
cudaStream_t ctx_stream(tpc_ctx *c);

}  // namespace tpc
