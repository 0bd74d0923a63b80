// nsn_internal.h -- declarations shared by the two translation units of the
// library (not part of the C ABI).
#ifndef NSN_INTERNAL_H
#define NSN_INTERNAL_H
#include <cuda_runtime.h>

#include "../../include/nsn.h"

// The stream all work of a collider is ordered on (defined with C linkage in
// nsn_collide.cu).
extern "C" cudaStream_t nsn_collider_stream_of(const nsn_collider *c);

#endif
