// Second pass (Sec. 6): once the detection step has run, every pixel is
// unmixed again with only the minerals detected in it and the additional
// spectra, which sharpens the abundances of the minerals that are there.
//
// Pixels are grouped by their detection mask on the host (one copy of the
// N masks, a stable sort of the pixel indices by mask); each group is
// gathered into a contiguous block (gather_kernel), unmixed by the full
// path on a handle for its sub-library, and its results are scattered
// back into the N x P outputs with zeros in the left-out columns
// (scatter_kernel, which also counts non-converged pixels).  Everything is
// queued on one stream; the handles are freed stream-ordered.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "api_internal.h"
#include "linmin.h"

namespace {

struct ColMap {
    int pos[LINMIN_MAX_P];   // column of the sub-problem holding column k, or -1
};

__global__ void gather_kernel(const float *__restrict__ cube, const long long *__restrict__ idx,
                              long long c, int L, float *__restrict__ out)
{
    const long long total = c * L;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / L;
        const int l = (int)(e - i * L);
        out[e] = cube[idx[i] * L + l];
    }
}

__global__ void scatter_kernel(const long long *__restrict__ idx, long long c, int P, int Pm,
                               ColMap map, const float *__restrict__ sx_sub,
                               const float *__restrict__ ssx_sub, const float *__restrict__ rms_sub,
                               const int *__restrict__ it_sub, float *x, float *sx, float *rms,
                               int *it, unsigned long long *n_bad)
{
    const long long total = c * P;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / P;
        const int k = (int)(e - i * P);
        const long long n = idx[i];
        const int p = map.pos[k];
        if (x) x[n * P + k] = p >= 0 ? sx_sub[i * Pm + p] : 0.f;
        if (sx) sx[n * P + k] = p >= 0 ? ssx_sub[i * Pm + p] : 0.f;
        if (k == 0) {
            if (rms) rms[n] = rms_sub[i];
            const int t = it_sub[i];
            if (it) it[n] = t;
            if (t < 0) atomicAdd(n_bad, 1ull);
        }
    }
}

int blocks_for(long long work)
{
    const long long b = (work + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 8));
}

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

// Stream-ordered scratch freed on every exit path.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> p;
    template <typename T>
    cudaError_t get(T **out, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(n, 1) * sizeof(T), s);
        if (e == cudaSuccess) p.push_back(q);
        *out = static_cast<T *>(q);
        return e;
    }
    ~Scratch()
    {
        for (void *q : p) cudaFreeAsync(q, s);
    }
};

}  // namespace

extern "C" linmin_status linmin_second_pass(const float *library, int L, int P, int n_minerals,
                                            const linmin_options *opt, const float *cube,
                                            long long N, const float *sigma,
                                            const unsigned long long *mask, float *abundances,
                                            float *uncertainties, float *residual_rms,
                                            int *iterations, int *n_groups)
{
    if (n_groups) *n_groups = 0;
    if (P < 1 || P > LINMIN_MAX_P || L < P || L > LINMIN_MAX_L)
        return sp_err(LINMIN_ERR_INVALID, "1 <= P <= 64 and P <= L <= 4096");
    if (n_minerals < 0 || n_minerals >= P)
        return sp_err(LINMIN_ERR_INVALID, "0 <= n_minerals < P (the additional spectra are always kept)");
    if (N < 0 || !library || (N > 0 && (!cube || !sigma || !mask)))
        return sp_err(LINMIN_ERR_INVALID, "library, cube, sigma and mask are required");
    const void *dev[] = {cube, sigma, mask, abundances, uncertainties, residual_rms, iterations};
    for (const void *p : dev)
        if (!device_or_null(p)) return sp_err(LINMIN_ERR_INVALID, "cube, sigma, mask and outputs must be device memory");
    linmin_options o;
    linmin_default_options(&o);
    if (opt) o = *opt;
    o.profile = 0;
    cudaStream_t s = static_cast<cudaStream_t>(o.cuda_stream);

    // the full library must give a unique minimiser; then so does every
    // subset of its columns (columns of a full-rank matrix stay independent)
    std::vector<float> hS;
    std::string why;
    linmin_status st = lm::load_library(library, L, P, &hS, &why);
    if (st != LINMIN_OK) return sp_err(st, why);
    if (N == 0) return LINMIN_OK;

    // group the pixels by mask
    std::vector<unsigned long long> hm((size_t)N);
    cudaError_t e = cudaMemcpyAsync(hm.data(), mask, (size_t)N * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sp_err(LINMIN_ERR_CUDA, cudaGetErrorString(e));
    const unsigned long long keep = n_minerals >= 64 ? ~0ull : ((1ull << n_minerals) - 1ull);
    for (auto &m : hm) m &= keep;
    std::vector<long long> order((size_t)N);
    std::iota(order.begin(), order.end(), 0LL);
    std::stable_sort(order.begin(), order.end(),
                     [&](long long a, long long b) { return hm[a] < hm[b]; });
    std::vector<long long> start;
    for (long long i = 0; i < N; ++i)
        if (i == 0 || hm[order[i]] != hm[order[i - 1]]) start.push_back(i);
    start.push_back(N);
    const int G = (int)start.size() - 1;
    long long cmax = 0;
    for (int g = 0; g < G; ++g) cmax = std::max(cmax, start[g + 1] - start[g]);

    Scratch sc{s, {}};
    long long *dIdx = nullptr;
    float *dY = nullptr, *dx = nullptr, *dsx = nullptr, *drms = nullptr;
    int *dit = nullptr;
    unsigned long long *dbad = nullptr;
    e = sc.get(&dIdx, (size_t)N);
    if (e == cudaSuccess) e = sc.get(&dY, (size_t)cmax * L);
    if (e == cudaSuccess) e = sc.get(&dx, (size_t)cmax * P);
    if (e == cudaSuccess) e = sc.get(&dsx, (size_t)cmax * P);
    if (e == cudaSuccess) e = sc.get(&drms, (size_t)cmax);
    if (e == cudaSuccess) e = sc.get(&dit, (size_t)cmax);
    if (e == cudaSuccess) e = sc.get(&dbad, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dIdx, order.data(), (size_t)N * sizeof(long long),
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sp_err(e == cudaErrorMemoryAllocation ? LINMIN_ERR_OOM : LINMIN_ERR_CUDA,
                      cudaGetErrorString(e));
    }

    std::vector<float> sub;
    for (int g = 0; g < G; ++g) {
        const long long off = start[g], c = start[g + 1] - start[g];
        const unsigned long long m = hm[order[off]];
        ColMap map;
        std::vector<int> cols;
        for (int k = 0; k < P; ++k) {
            const bool kept = k >= n_minerals || ((m >> k) & 1ull);
            map.pos[k] = kept ? (int)cols.size() : -1;
            if (kept) cols.push_back(k);
        }
        for (int k = P; k < LINMIN_MAX_P; ++k) map.pos[k] = -1;
        const int Pm = (int)cols.size();
        sub.assign((size_t)Pm * L, 0.f);
        for (int r = 0; r < Pm; ++r)
            std::copy(hS.begin() + (size_t)cols[r] * L, hS.begin() + (size_t)(cols[r] + 1) * L,
                      sub.begin() + (size_t)r * L);
        linmin_handle hs = nullptr;
        st = linmin_create(sub.data(), L, Pm, &o, &hs);
        if (st != LINMIN_OK)
            return sp_err(st, std::string("sub-library handle: ") + linmin_last_error(nullptr));
        gather_kernel<<<blocks_for(c * L), 256, 0, s>>>(cube, dIdx + off, c, L, dY);
        st = linmin_unmix(hs, dY, c, sigma, dx, dsx, drms, dit);
        if (st != LINMIN_OK && st != LINMIN_ERR_NOT_CONVERGED) {
            const std::string m2 = linmin_last_error(hs);
            lm::destroy_async(hs);
            return sp_err(st, m2);
        }
        scatter_kernel<<<blocks_for(c * P), 256, 0, s>>>(dIdx + off, c, P, Pm, map, dx, dsx, drms,
                                                         dit, abundances, uncertainties,
                                                         residual_rms, iterations, dbad);
        lm::destroy_async(hs);
        e = cudaGetLastError();
        if (e != cudaSuccess) return sp_err(LINMIN_ERR_CUDA, cudaGetErrorString(e));
    }
    unsigned long long nbad = 0;
    e = cudaMemcpyAsync(&nbad, dbad, sizeof(nbad), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sp_err(LINMIN_ERR_CUDA, cudaGetErrorString(e));
    if (n_groups) *n_groups = G;
    return nbad ? LINMIN_ERR_NOT_CONVERGED : LINMIN_OK;
}
