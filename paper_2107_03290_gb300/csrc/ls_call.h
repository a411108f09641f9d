// Host-side interface between the C ABI entry points, the server and the sort
// path: how one call reports its asynchronous errors.  Plain C++, shared by
// the CUDA translation units and the server.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include "../../include/ls.h"

struct CUstream_st;

namespace ls {

// Status block of one call (or one server request), in device memory.
// Kernels receive a pointer to `word` (the first member) as `uint32_t* err`
// and record ERR_* bits there; the other fields steer the bounded waits.  Each
// call zeroes its own block at its start, so that an earlier call's error
// never stops a later one, and ORs the word into a persistent block (the
// stream's, or a server request's) at its end.
struct CallStatus {
  uint32_t word;                  // ERR_* bits
  uint32_t stall;                 // STALL_* test injection (0 in normal use)
  unsigned long long spin_limit;  // polls before a wait gives up (0: the default)
};

// Where a call's errors go and the test settings of its bounded waits.
struct CallOpts {
  CallStatus* fold_to;            // device address of the persistent block
  uint32_t stall;
  unsigned long long spin_limit;
};

// ls_sort_ex / ls_sort_batch with an explicit error destination (the server's
// per-request blocks).  `o` == nullptr: the stream's persistent block.
ls_status sort_call(void* keys, size_t n, ls_dtype dtype, CUstream_st* stream,
                    const ls_params* params, ls_stats* stats, const CallOpts* o);
ls_status batch_call(void* const* keys, const size_t* n, size_t count, ls_dtype dtype,
                     CUstream_st* stream, const CallOpts* o, const ls_batch_params* bp = nullptr);

// Scratch from the library's per-device stream-ordered memory pool (the one
// every sort call carves its workspace from).  pool_alloc returns 0 on
// success, else a CUDA error code; pool_free releases in stream order.
int pool_alloc(void** p, size_t bytes, CUstream_st* stream);
void pool_free(void* p, CUstream_st* stream);

}  // namespace ls
