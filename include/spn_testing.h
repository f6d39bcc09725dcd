/*
 * spn_testing.h -- test support of libspn, kept apart from the product API of
 * spn.h.  Nothing here is needed to run simulations; the paper has no
 * counterpart.
 */
#ifndef SPN_TESTING_H
#define SPN_TESTING_H

#include <stdint.h>

#include "spn.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Failure detection without a device fault.  Arms handle h (an Ising lattice)
 * only: in its next streaming-sweep launch the copy of each CTA's first slice is
 * never issued, so the wait for it runs out after `polls` polls (0 counts as 1).
 * The kernel then records the failure, waits (with the full bound) for the
 * copies it did issue and returns; no device fault occurs, the context stays
 * usable, and the next spn_observables / spn_trace / spn_sync of that handle
 * returns SPN_E_TIMEOUT.  Launches of other handles are unaffected.  The arming
 * is consumed by that launch; a handle that never runs a streaming launch keeps
 * it until it is destroyed.  Returns SPN_E_STATE for a batch or Heisenberg
 * handle. */
int spn_test_expire_next_waits(spn_handle h, uint32_t polls);

#ifdef __cplusplus
}
#endif

#endif /* SPN_TESTING_H */
