/*
 * sbp_check.h -- test entry points of libsbp that need no device: host
 * runs of device-side logic, compared with the host code it must follow.
 * Conventions as in sbp.h (SBP_OK or a negative SBP_E* code, the message
 * through sbp_last_error, host arrays borrowed for the call).
 */
#ifndef SBP_CHECK_H
#define SBP_CHECK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The golden-ratio search over the number of blocks (Section II-B) as the
 * batching form's persistent kernel runs it, compiled for and run on the
 * host, against the host driver's bracket: the states (B[i] >= 1, dl[i]) are
 * inserted in order into both; after each insert, out[12 i + 0..5] holds the
 * host bracket's three position B values (0: empty), whether a next phase
 * exists, its start position and target, and out[12 i + 6..11] the same
 * from the kernel's copy (host arrays, count * 12 entries).  *n_bad counts
 * the steps where the two differ or the kernel's label slots collide.
 * reduction: (0, 1), as in sbp_params.  SBP_EINVAL on a negative count, a
 * NULL array, B[i] < 1 or a reduction outside (0, 1). */
int sbp_bracket_check(const int32_t *B, const double *dl, int32_t count, double reduction, int32_t *out,
                      int32_t *n_bad);

#ifdef __cplusplus
}
#endif

#endif /* SBP_CHECK_H */
