// Internal device-wide primitives (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace lt {

// Exclusive prefix sum of `count` uint32 values (the total must fit in 32
// bits); `in` and `out` may alias.  `tmp` needs scan_tmp_words(count) words.
size_t scan_tmp_words(int64_t count);
cudaError_t scan_u32_exclusive(const uint32_t* in, uint32_t* out, int64_t count, uint32_t* tmp,
                               cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the
// key, 8 bits per pass.  Ping-pongs between (k0, v0) and (k1, v1); returns in
// *in_alt whether the result ended in (k1, v1).  `hist` needs
// radix_hist_words(count) words, `tmp` scan_tmp_words(radix_hist_words(count)).
size_t radix_hist_words(int64_t count);
cudaError_t radix_sort_u64_f64(uint64_t* k0, double* v0, uint64_t* k1, double* v1, int64_t count, int bits,
                               uint32_t* hist, uint32_t* tmp, cudaStream_t s, bool* in_alt);

// The same for keys alone, by bits [lo_bit, lo_bit + bits) of the key (the
// bits below lo_bit travel with the key unsorted).
cudaError_t radix_sort_u64(uint64_t* k0, uint64_t* k1, int64_t count, int lo_bit, int bits, uint32_t* hist,
                           uint32_t* tmp, cudaStream_t s, bool* in_alt);

size_t bfs_warp_bytes(int k, int* hlog2_out);

}  // namespace lt
