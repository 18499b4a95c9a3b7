/*
 * scoup_selftest.h -- self-tests and measurement helpers of libscoup.so.
 * The paper has no counterpart to either: the first checks the library's own
 * guard that a tensor-core pipeline wait which never completes gives up,
 * reports an error and leaves the GPU usable, without faulting anything; the
 * second measures the GPU's atomic-update ceiling that bounds the uplift's
 * scatter (Eq. 5), for the roofline of the uplift step.
 */
#ifndef SCOUP_SELFTEST_H
#define SCOUP_SELFTEST_H

#include <stddef.h>
#include <stdint.h>

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

/* Atomic-update throughput: `count` FP32 atomic additions (reductions whose
 * result is not read, like the uplift's accumulator updates) of 1.0 to
 * pseudo-random elements of buf, spread uniformly over its first 2^log2_n
 * floats (a hash of the update index and `seed` picks the element).
 *  buf       DEVICE, >= 2^log2_n floats (4 * 2^log2_n bytes), caller-owned;
 *            its values are changed (each element grows by the number of
 *            updates it received).
 *  log2_n    in [10, 31].
 *  count     >= 0 updates.
 * Enqueued on `stream` without synchronising; time it with events on that
 * stream.  Returns SCOUP_ERR_INVALID_ARG on a bad argument, SCOUP_ERR_CUDA on a
 * launch error. */
int scoup_selftest_red_throughput(float* buf, int32_t log2_n, int64_t count, uint32_t seed, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SCOUP_SELFTEST_H */
