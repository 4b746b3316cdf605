// Index checks of the bounds-check build (compiled with -DTF_BOUNDS_CHECK into
// libtwofluid_bc.so; a stand-in for a memory checker).  Every checked index
// that falls outside its extent sets a per-CTA flag and is replaced by 0, so
// the access stays in bounds; at the end of the kernel thread 0 records
// TF_ERR_BOUNDS in the context's status word, which tf_sync returns.  Nothing
// traps.  In the normal build the checks compile to nothing.
#pragma once

#include "tf_internal.h"

#ifdef TF_BOUNDS_CHECK
__device__ __forceinline__ int* tf_bc_flag() {
    __shared__ int flag;
    return &flag;
}
// Start of a kernel: clear the flag (contains a CTA barrier).
__device__ __forceinline__ void tf_bc_begin() {
    if (threadIdx.x == 0) *tf_bc_flag() = 0;
    __syncthreads();
}
__device__ __forceinline__ long long tf_bc(long long i, long long n) {
    if (i < 0 || i >= n) {
        *tf_bc_flag() = 1;
        return 0;
    }
    return i;
}
// End of a kernel (every thread, all paths): report the flag.
__device__ __forceinline__ void tf_bc_end(int* err) {
    __syncthreads();
    if (threadIdx.x == 0 && *tf_bc_flag()) atomicCAS(err, 0, TF_ERR_BOUNDS);
}
#define TF_BC(i, n) ((int)tf_bc((i), (n)))
#define TF_BC64(i, n) tf_bc((i), (n))
#define TF_BC_BEGIN() tf_bc_begin()
#define TF_BC_END(err) tf_bc_end(err)
#else
#define TF_BC(i, n) (i)
#define TF_BC64(i, n) (i)
#define TF_BC_BEGIN() ((void)0)
#define TF_BC_END(err) ((void)0)
#endif
