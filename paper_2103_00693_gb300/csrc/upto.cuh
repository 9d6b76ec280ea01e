// Launchers of the small-instance store and reduce (upto.cu): every solution
// of a handle up to a cap, with the rank read on the device.
#pragma once

#include "hlf_internal.cuh"

namespace hlf {

// out[i][0..W) = z(i) for i < min(2^r, cap), r = info[1] as the factor
// kernel left it (nothing is written when r < 0). out: 8-byte aligned.
hlf_status launch_store_upto(const uint64_t* table, int W, const int32_t* info, uint64_t cap, uint64_t* out,
                             cudaStream_t s);

// *out (zeroed by the caller) += the reduce of [0, min(2^r, cap)); nothing is
// added when r < 0.
hlf_status launch_reduce_upto(const uint64_t* table, int W, const int32_t* info, uint64_t cap, hlf_reduce* out,
                              cudaStream_t s);

}  // namespace hlf
