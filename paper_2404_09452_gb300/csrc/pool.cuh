// Device memory cache of the DF-J/K library (pool.cu): blocks released by a
// handle are kept per device and size and handed to the next request of the
// same size, so repeated setups and builds of similar molecules do not pay
// cudaMalloc/cudaFree (which synchronise the device) every time.
#pragma once

#include <stddef.h>

namespace dfjk {

void *pool_alloc(size_t bytes);          // throws Error{DFJK_ERR_OOM} on failure
void pool_free(void *p, size_t bytes);   // returns the block to the cache
void pool_trim();                        // frees every cached block of this device
size_t pool_cached_bytes();

}  // namespace dfjk
