/*
 * scoup_selftest.h -- self-test of the device-side failure detection of
 * libscoup.so.  The paper has no counterpart: this checks the library's own
 * guard that a tensor-core pipeline wait which never completes gives up,
 * reports an error and leaves the GPU usable, without faulting anything.
 */
#ifndef SCOUP_SELFTEST_H
#define SCOUP_SELFTEST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Launches a 128 x 64 x 64 codebook-decode GEMM (the tcgen05 kernel of
 * scoup_decode) whose load warp issues no copies, so the MMA and epilogue
 * warps' bounded mbarrier waits (about 2^22 polls, well under a second) run
 * out.  The kernel records the timeout in its status word, frees its TMEM
 * and returns; the call synchronises `stream`.
 *  workspace  DEVICE, >= 49408 bytes, 256-byte aligned (overwritten).
 * Returns SCOUP_ERR_TIMEOUT when the guard worked (the expected result),
 * SCOUP_ERR_DEVICE_CHECK if no timeout was reported, another error if the
 * test could not run.  The context stays usable afterwards. */
int scoup_selftest_gemm_timeout(void* workspace, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SCOUP_SELFTEST_H */
