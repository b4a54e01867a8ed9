// Internal entry points shared by the C ABI translation units (not exported).
#pragma once
#include <string>
#include <vector>

#include "linmin.h"

namespace lm {

// Copy a P x L library (host or device pointer) to *host and check it:
// finite values and rank [S^T; 1^T] = P.  *why receives the reason of a
// failure.
linmin_status load_library(const float *library, int L, int P, std::vector<float> *host,
                           std::string *why);

// A handle for a library already loaded and checked by load_library, with
// validated options (no checks of its own).
linmin_status create_from_host(const float *host_library, int L, int P,
                               const linmin_options &opt, linmin_handle *out);

// Free a handle without synchronising: its device memory returns to the
// pool once the work already queued on its stream has run.
linmin_status destroy_async(linmin_handle h);

// Device bytes a handle for (L, P) holds once reserved for N pixels (with
// the host-pointer staging buffers when host_io).
size_t handle_bytes(int L, int P, long long N, bool host_io);

// Allocate a handle's per-pixel scratch (and staging) for N pixels now, so
// that later calls with at most N pixels allocate nothing.
linmin_status reserve(linmin_handle h, long long N, bool host_io);

// Record the message linmin_last_error(NULL) returns (entry points
// without a handle).
void set_global_error(const std::string &m);

// N >= 1 when LINMIN_FAIL_ALLOC = N asks for the N-th device allocation of
// a handle (or of a call that allocates on its own) to fail; else 0.
long long injected_alloc_failure();

}  // namespace lm
