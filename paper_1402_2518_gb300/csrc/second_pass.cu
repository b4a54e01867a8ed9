// Second pass (Sec. 5): once the detection step has run, every pixel is
// unmixed again with only the minerals detected in it and the additional
// spectra, which sharpens the abundances of the minerals that are there.
//
// One handle for the full library and one linmin_unmix_masked call: the
// left-out minerals of each pixel are removed by an exact linear penalty
// on their projections (launch_exclude), so all pixels, whatever their
// subsets, go through the same launches as a plain unmixing.
#include <cuda_runtime.h>

#include <string>

#include "api_internal.h"
#include "linmin.h"

namespace {

linmin_status sp_err(linmin_status st, const std::string &m)
{
    lm::set_global_error("linmin_second_pass: " + m);
    return st;
}

bool device_or_null(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" linmin_status linmin_second_pass(const float *library, int L, int P, int n_minerals,
                                            const linmin_options *opt, const float *cube,
                                            long long N, const float *sigma,
                                            const unsigned long long *mask, float *abundances,
                                            float *uncertainties, float *residual_rms,
                                            int *iterations)
{
    if (P < 1 || P > LINMIN_MAX_P || L < P || L > LINMIN_MAX_L)
        return sp_err(LINMIN_ERR_INVALID, "1 <= P <= 64 and P <= L <= 4096");
    if (n_minerals < 0 || n_minerals >= P)
        return sp_err(LINMIN_ERR_INVALID, "0 <= n_minerals < P (the additional spectra are always kept)");
    if (N < 0 || !library || (N > 0 && (!cube || !sigma || !mask)))
        return sp_err(LINMIN_ERR_INVALID, "library, cube, sigma and mask are required");
    const void *dev[] = {cube, sigma, mask, abundances, uncertainties, residual_rms, iterations};
    for (const void *p : dev)
        if (!device_or_null(p))
            return sp_err(LINMIN_ERR_INVALID, "cube, sigma, mask and outputs must be device memory");
    if (N == 0) return LINMIN_OK;
    linmin_options o;
    linmin_default_options(&o);
    if (opt) o = *opt;
    o.profile = 0;
    linmin_handle h = nullptr;
    linmin_status st = linmin_create(library, L, P, &o, &h);
    if (st != LINMIN_OK) return sp_err(st, linmin_last_error(nullptr));
    st = linmin_unmix_masked(h, cube, N, sigma, mask, n_minerals, abundances, uncertainties,
                             residual_rms, iterations);
    if (st == LINMIN_OK) st = linmin_wait(h, nullptr);
    std::string m = st == LINMIN_OK || st == LINMIN_ERR_NOT_CONVERGED ? "" : linmin_last_error(h);
    linmin_destroy(h);
    if (!m.empty()) return sp_err(st, m);
    return st;
}
