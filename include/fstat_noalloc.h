/*
 * fstat_noalloc.h -- a toplist call that allocates no device memory (part of
 * libfstat.so).
 *
 * The paper has no counterpart to this call: it is a library convenience.
 * fstat_compute keeps its toplist scratch in buffers the context allocates.
 * Some callers cannot let a library allocate at the point of the call: a
 * process whose device memory is all handed out by its own pool or caching
 * allocator, a latency-bound loop that cannot take the device-wide
 * synchronisation that freeing device memory implies, or code that must not
 * fail with out-of-memory halfway through a step.  For them this call ranks a
 * 2F array that already lives on the device, with every intermediate held in
 * one fixed scratch area compiled into the library (one per device).
 */
#ifndef FSTAT_NOALLOC_H
#define FSTAT_NOALLOC_H

#include <stdint.h>

#include "fstat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest k the call accepts; the scratch area is sized for it:
 * 3 x 2048 histogram words, 16 state words, 1024 block tie counts, one slot
 * counter and k (index, value) candidate slots = 225,348 bytes, rounded up to
 * 225,536 (a multiple of 256). */
#define FSTAT_NOALLOC_MAX_K 16384

/* The k largest values of v[0 .. n-1] (device FP32, n >= 1, values >= 0 and
 * not NaN as 2F is; -0.0 ranks as +0.0 and is returned as +0.0), ordered by
 * value descending and, for equal values, by index ascending -- the order
 * fstat_get_toplist returns.  idx_out [k] (int64) and val_out [k] (FP32) are
 * device arrays owned by the caller.
 *
 * Alignment: v may start at any element (4-byte aligned address, e.g. a view
 * at an offset into a larger array); val_out must be 4-byte and idx_out
 * 8-byte aligned.  A pointer that breaks this is refused with EINVAL before
 * anything is launched.
 *
 * Everything runs asynchronously on cuda_stream (NULL = the legacy default
 * stream) on `device`, which becomes the calling thread's current device.
 *
 * Scratch: a static device array of the size above.  Its histogram, state and
 * slot-counter words must start at zero for each call; the call clears them
 * itself with cudaMemsetAsync on cuda_stream before its first kernel, so the
 * caller has nothing to prepare and may rely on nothing it leaves behind.
 * Because there is one scratch area per device, calls on the same device whose
 * executions can overlap (on different streams, or from different host
 * threads without ordering) race on it and give wrong results: order them, for
 * example by issuing them on one stream.
 *
 * Setup: the first call on each device looks up the scratch area's address
 * with cudaGetSymbolAddress (this may load the library's device code on that
 * device) and keeps it for later calls; make that first call before any
 * stream capture begins.
 *
 * msg / msg_len (optional, may be NULL / 0): receives a one-line description
 * of an error.  Errors: ERANGE (k above FSTAT_NOALLOC_MAX_K), EINVAL (null or
 * misaligned pointers, n < 1, k < 1 or k > n, bad device), ECUDA (a CUDA call
 * failed). */
int fstat_toplist_noalloc(int device, const float *v, int64_t n, int32_t k, int64_t *idx_out, float *val_out,
                          void *cuda_stream, char *msg, int32_t msg_len);

#ifdef __cplusplus
}
#endif
#endif /* FSTAT_NOALLOC_H */
