// Batched primal-dual interior-point FCLS solve (IPLS, Sec. 2.2) on sm_103a.
//
// Problem per pixel, in the scaled units set by the library preparation
// (G~ = G / s + rho 1 1^T, c~ = c / s + rho 1, s = trace(G) / P, rho = 1):
//
//     minimise 1/2 x^T G~ x - c~^T x   s.t.  x >= 0,  1^T x = 1
//
// Adding rho 1 1^T to G and rho 1 to c changes nothing on the feasible set
// (the added term rho/2 (1^T x - 1)^2 vanishes there), so the minimiser is
// the FCLS one of eqs. NonNegativity/SumToOne; it makes every barrier
// Hessian H = G~ + X^-1 Lambda positive definite when rank [S^T; 1^T] = P
// even though G itself is singular for the level/slope spectra of Sec. 2.5
// (flat, increasing and decreasing slopes are linearly dependent).
//
// Each Newton step solves the bordered KKT system
//     [ H   1 ] [dx ]   [ -r_d - X^-1 r_c ]
//     [ 1^T 0 ] [dnu] = [ -r_p            ]
// through H = L L^T and u = H^-1 1: dnu = (1^T H^-1 r + r_p) / (1^T u),
// dx = H^-1 (r - dnu 1); only forward solves are needed for the scalars
// (1^T H^-1 r = (L^-1 1).(L^-1 r)), one back solve per direction.  The
// step is Mehrotra's predictor-corrector with a common primal/dual step
// length (fraction to the boundary eta).
//
// Mapping: a group of G consecutive lanes owns one pixel; lane t owns rows
// i = s*G + t (slot s < NS) of the lower triangle of H, kept in registers
// (row length (s+1)*G, fully unrolled, compile-time indices).  The
// factorisation is right-looking and leaves the columns of L in shared
// memory, where the triangular solves read them; the right-hand sides 1 and
// r_aff are eliminated during the factorisation (forward solves for free).
//   * G = 4: by blocks of four columns (one slot).  Every lane of the group
//     factors the 4 x 4 diagonal block itself (its rows exchanged through
//     shared memory), forms its own panel rows in place and updates the
//     trailing rows with a rank-4 update in packed FMAs (fma.rn.f32x2):
//     every register index is a compile-time constant, so there are no
//     selects or predicated updates.
//   * G > 4: column by column, the G columns of a slot sharing one copy of
//     the code (a rolled loop, the column picked by selects), which keeps
//     the loop body of the wider groups small.
// The solves go by blocks of G rows through the inverses of the diagonal
// blocks of L (stored in place of those blocks): one gather of G values by
// shuffles per block instead of one broadcast per row, and every shared
// memory address of the column reads a compile-time offset.  Groups take
// pixels from a global work counter and refill as soon as their pixel
// leaves the active set (converged pixels are compacted out of the running
// set; warps run while any group has work).
//
// Two instantiations per size: ACC = false iterates with the float32 KKT
// residual until mu <= mu_ref and saves the state; ACC = true continues with
// the residual G~ x - c~ evaluated in double-float (G~ and c~ as hi+lo
// float32 pairs) until the stopping test, so the iterates converge to the
// minimiser of the exact data rather than of its float32 rounding.
#pragma once
#include "common.cuh"
#include <type_traits>

namespace lm {


// Compiler-only memory fence: keeps the scheduler from hoisting the shared
// memory loads of later unrolled steps (which would hold them all in
// registers at once).
#define LM_STEP_FENCE() asm volatile("" ::: "memory")


// two FMAs in one instruction: (d0, d1) = (a0 * b0 + c0, a1 * b1 + c1), operands
// passed as scalars so that the register arrays stay scalarisable
LM_DEV void ffma2s(float &d0, float &d1, float a0, float a1, float b0, float b1, float c0, float c1)
{
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d0), "=f"(d1) : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(c0), "f"(c1));
}

// compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1
template <int I, int N, typename F>
LM_DEV void lm_static_for_impl(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        lm_static_for_impl<I + 1, N>(f);
    }
}
template <int N, typename F>
LM_DEV void lm_static_for(F &&f) { lm_static_for_impl<0, N>(f); }

// One cube of a batched launch (sum-to-one handles of the same P): its
// scaled projection, its G~ and start gradient in global memory, its state
// arrays, and the first global work index of its pixels.
struct IpmCube {
    long long N, start;
    const float *c_hi;             // N x P
    const float *Ghi, *grs;        // PP x PP (zero padded), PP
    float *x_state, *lam_state, *nu_state;
    int *it_state;
};

struct IpmArgs {
    long long N;
    int P;
    int max_iter;
    const float *c_hi, *c_lo;      // N x P, scaled projection c~ (hi + lo)
    const float *Ghi, *Glo;        // PP x PP row-major, zero padded (G~ hi + lo)
    const float *grs;              // PP: G~ x0, the gradient term at the start x0
    int slack_idx = -1;            // x0: 1/P, or slack_x0 on slack_idx and
    float slack_x0 = 0.f;          //     (1 - slack_x0) / (P - 1) elsewhere
    float *x_state, *lam_state;    // N x P
    float *nu_state;               // N
    int *it_state;                 // N: iterations so far (phase A) / final (phase B, <0: cap)
    unsigned long long *counter;   // pixel work counter, zeroed before the launch
    unsigned long long *n_notconv; // phase B: number of pixels that hit max_iter
    const long long *list;         // optional: pixels to process (else 0..N-1)
    const unsigned long long *list_len;  // number of entries of list
    float mu_ref, tol_c, tol_d, eta;
    // batched launch (BATCH kernels): one work counter over the pixels of
    // n_cubes cubes, total = their pixel count; the other per-cube fields
    // above are unused
    const IpmCube *cubes = nullptr;
    int n_cubes = 0;
    unsigned long long total = 0;
};

template <int NS_, int G_>
struct IpmCfg {
    static constexpr int NS = NS_, G = G_;
    static constexpr int PP = NS * G;      // padded size, multiple of 4
    static constexpr int GPW = 32 / G;     // pixel groups per warp
    // registers of H per lane (rows of (s+1)*G floats)
    static constexpr int H_REGS = NS * (NS + 1) / 2 * G;
    // Warps per block and the resident blocks per SM the register budget is
    // sized for.  Four- and eight-lane groups run the block-panel
    // factorisation, whose unrolled loop body is large: eight warps per block
    // iterate in lockstep, so the two warps of each scheduler fetch the same
    // instructions (four lanes: one 8-warp block per SM above 100 registers
    // of H, else 2; eight lanes: one).  Sixteen-lane groups keep 4-warp
    // blocks (2 per SM above 100 registers of H, else 3).
    static constexpr int WARPS = (G <= 8) ? 8 : 4;
    static constexpr int MIN_BLOCKS = (G == 4) ? (H_REGS > 100 ? 1 : 2) : (G == 8 ? 1 : (H_REGS > 100 ? 2 : 3));
    static constexpr int THREADS = WARPS * 32;
    // column k of L is stored for rows alignrow(k) .. PP-1 (16-byte aligned)
    static constexpr __host__ __device__ int alignrow(int k) { return ((k + 1) / 4) * 4; }
    static constexpr __host__ __device__ int collen(int k) { return PP - alignrow(k); }
    // sum_{q<k} collen(q) = k*PP - 4*sum_{m=1..k} floor(m/4), in closed form
    // (cheap when k is a runtime row index)
    static constexpr __host__ __device__ int colstart(int k) {
        const int A = k / 4;
        return k * PP - 4 * (2 * A * (A - 1) + A * (k - 4 * A + 1));
    }
    // offset of column k's storage such that L[i][k] = buf[coloff(k) + i]
    static constexpr __host__ __device__ int coloff(int k) { return colstart(k) - alignrow(k); }
    static constexpr int LBUF = colstart(PP);
    // per-group floats: L columns + a broadcast area (x in the residual, the
    // diagonal block rows in the factorisation: at least 32 floats); stride
    // = G (mod 32) words, so that the G consecutive words the lanes of each
    // group read or write at one offset (solves, panel stores) fall in
    // distinct banks for the GPW groups of a warp
    static constexpr int GROUP_RAW = LBUF + (PP > 32 ? PP : 32);
    static constexpr int GROUP_FLOATS = ((GROUP_RAW + 31) / 32) * 32 + G;
    // row stride of G~ in shared memory: 4 (mod 8) words, so that the rows
    // of consecutive lanes (read at the same column with LDS.128) start 4,
    // 12, 20 or 28 banks apart and up to eight of them share no bank
    static constexpr int GS = (PP % 8 == 4) ? PP : PP + 4;
    static constexpr size_t smem_bytes(bool acc) {
        return sizeof(float) * ((acc ? 2 : 1) * PP * GS + PP +
                                (size_t)WARPS * GPW * GROUP_FLOATS);
    }
};

template <int NS, int G, bool ACC, bool BATCH = false>
__global__ void __launch_bounds__(IpmCfg<NS, G>::THREADS, IpmCfg<NS, G>::MIN_BLOCKS)
ipm_kernel(const IpmArgs a)
{
    static_assert(!(ACC && BATCH), "batched launches run the float32 phase");
    using C = IpmCfg<NS, G>;
    constexpr int PP = C::PP;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr float TINY = 1e-30f, BIGPIV = 1e30f, DMAX = 1e30f;

    extern __shared__ __align__(16) float sm[];
    float *sGhi = sm;                                // PP rows of C::GS words
    float *sGlo = sm + PP * C::GS;                   // only with ACC
    float *sGrs = sm + (ACC ? 2 : 1) * PP * C::GS;
    float *grp0 = sGrs + PP;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = lane % G, gid = lane / G;
    const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (gid * G));
    float *colbuf = grp0 + (warp * C::GPW + gid) * C::GROUP_FLOATS;
    float *xbuf = colbuf + C::LBUF;

    if constexpr (!BATCH) {
        for (int e = threadIdx.x; e < PP * PP; e += blockDim.x) {
            const int r = e / PP, q = e - r * PP;
            sGhi[r * C::GS + q] = a.Ghi[e];
            if (ACC) sGlo[r * C::GS + q] = a.Glo[e];
        }
        for (int e = threadIdx.x; e < PP; e += blockDim.x) sGrs[e] = a.grs[e];
    }
    __syncthreads();
    // G~ rows: shared memory, or (batch) the group's current cube in global
    // memory (read through L1)
    const float *gG = sGhi;
    constexpr int GST = BATCH ? PP : C::GS;          // row stride of gG's rows
    const IpmCube *cb = nullptr;
    auto ldG4 = [&](const float *q) -> float4 {
        if constexpr (BATCH) return __ldg(reinterpret_cast<const float4 *>(q));
        else return *reinterpret_cast<const float4 *>(q);
    };

    const int P = a.P;
    const float invP = 1.0f / (float)P;
    const float x0o = a.slack_idx >= 0 ? (1.0f - a.slack_x0) / (float)(P - 1) : invP;
    bool valid[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) valid[s] = s * G + t < P;

    float x[NS], lam[NS], nu = 0.f;
    int it = 0;
    size_t cbase = 0;   // offset of the current pixel in the N x P arrays

    // pixel work list: 0..N-1, or the first list_len entries of list
    const unsigned long long n_work = a.list ? *a.list_len : (unsigned long long)a.N;
    // "no more work": a.N, or -1 in a batch
    auto has = [&](long long p) -> bool { return BATCH ? p >= 0 : p < a.N; };
    auto fetch = [&]() -> long long {
        if constexpr (BATCH) {
            // one counter over all cubes; the cube of a work index by
            // binary search over their first indices
            long long p = -1;
            int c = 0;
            if (t == 0) {
                const unsigned long long v = atomicAdd(a.counter, 1ULL);
                if (v < a.total) {
                    int lo = 0, hi = a.n_cubes - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((unsigned long long)a.cubes[mid].start <= v) lo = mid; else hi = mid - 1;
                    }
                    c = lo;
                    p = (long long)v - a.cubes[lo].start;
                }
            }
            p = __shfl_sync(gmask, p, 0, G);
            c = __shfl_sync(gmask, c, 0, G);
            cb = a.cubes + c;
            gG = cb->Ghi;
            return p;
        } else {
            unsigned long long v = 0;
            long long p = a.N;                      // a.N marks "no more work"
            if (t == 0) {
                v = atomicAdd(a.counter, 1ULL);
                if (v < n_work) p = a.list ? a.list[v] : (long long)v;
            }
            return __shfl_sync(gmask, p, 0, G);
        }
    };
    auto chi = [&]() -> const float * { if constexpr (BATCH) return cb->c_hi; else return a.c_hi; };

    // load c~ and either the start point (phase A) or the saved state (B)
    auto load_pixel = [&](long long p) {
        const size_t base = (size_t)p * P;
        cbase = base;
        if (!ACC) {
            // x0 (1/P, or the slack start); g0 = G~ x0 - c~; nu0 makes lambda0 = g0 + nu0 dual
            // feasible with min lambda0 = 1e-3 (a smaller start than adding
            // the spread of g0 as well: 11.2 instead of 11.7 iterations on
            // the OMEGA-shaped workload)
            float gmin = 3.4e38f, g0[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float gr = BATCH ? __ldg(cb->grs + s * G + t) : sGrs[s * G + t];
                g0[s] = valid[s] ? gr - __ldg(chi() + base + s * G + t) : 0.f;
                if (valid[s]) gmin = fminf(gmin, g0[s]);
            }
            for (int off = 1; off < G; off <<= 1)
                gmin = fminf(gmin, __shfl_xor_sync(gmask, gmin, off));
            nu = 1e-3f - gmin;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                x[s] = valid[s] ? (s * G + t == a.slack_idx ? a.slack_x0 : x0o) : 0.f;
                lam[s] = valid[s] ? g0[s] + nu : 0.f;
            }
            it = 0;
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int i = s * G + t;
                x[s] = valid[s] ? a.x_state[base + i] : 0.f;
                lam[s] = valid[s] ? a.lam_state[base + i] : 0.f;
            }
            nu = a.nu_state[p];
            it = a.it_state[p];
        }
    };

    long long pix = fetch();
    bool alive = has(pix);
    if (alive) load_pixel(pix);
    else {
#pragma unroll
        for (int s = 0; s < NS; ++s) { x[s] = valid[s] ? invP : 0.f; lam[s] = valid[s] ? 1.f : 0.f; }
    }

    float rd[NS];
    float rp = 0.f, mu = 0.f, rdmax = 0.f, dec = 0.f;

    // r_d = G~ x - c~ - lambda + nu 1 and the scalar measures (group-uniform).
    // G~ x is accumulated column by column in one sequential chain per row:
    // the pos thresholds sit at the float32 floor, and an even/odd split of
    // the sum (two packed chains) doubled pos's iteration count.
    auto residual = [&]() {
#pragma unroll
        for (int s = 0; s < NS; ++s) xbuf[s * G + t] = x[s];
        __syncwarp();
        if (!ACC) {
            // c~ loads issued first: their latency overlaps the dot products
            float acc[NS], cc[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                acc[s] = 0.f;
                cc[s] = valid[s] ? __ldg(chi() + cbase + s * G + t) : 0.f;
            }
#pragma unroll 1
            for (int j4 = 0; j4 < PP / 4; ++j4) {
                const float4 xv = *reinterpret_cast<const float4 *>(xbuf + 4 * j4);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const float4 g = ldG4(gG + (s * G + t) * GST + 4 * j4);
                    acc[s] = fmaf(g.x, xv.x, acc[s]);
                    acc[s] = fmaf(g.y, xv.y, acc[s]);
                    acc[s] = fmaf(g.z, xv.z, acc[s]);
                    acc[s] = fmaf(g.w, xv.w, acc[s]);
                }
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const float gx = acc[s] - cc[s];
                rd[s] = valid[s] ? (gx - lam[s]) + nu : 0.f;
            }
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int i = s * G + t;
                const float *grow = sGhi + i * C::GS;
                const float *glow = sGlo + i * C::GS;
                dot2 d;
#pragma unroll
                for (int j4 = 0; j4 < PP / 4; ++j4) {
                    const float4 g = *reinterpret_cast<const float4 *>(grow + 4 * j4);
                    const float4 gl = *reinterpret_cast<const float4 *>(glow + 4 * j4);
                    const float4 xv = *reinterpret_cast<const float4 *>(xbuf + 4 * j4);
                    d.add_prod(g.x, xv.x); d.c = fmaf(gl.x, xv.x, d.c);
                    d.add_prod(g.y, xv.y); d.c = fmaf(gl.y, xv.y, d.c);
                    d.add_prod(g.z, xv.z); d.c = fmaf(gl.z, xv.z, d.c);
                    d.add_prod(g.w, xv.w); d.c = fmaf(gl.w, xv.w, d.c);
                }
                if (valid[s]) d.add_df(df{-__ldg(a.c_hi + cbase + i), -__ldg(a.c_lo + cbase + i)});
                const df r = d.result();
                const float gx = r.hi + r.lo;
                rd[s] = valid[s] ? (gx - lam[s]) + nu : 0.f;
                LM_STEP_FENCE();
            }
        }
        __syncwarp();
        float sx = 0.f, sxl = 0.f, rmax = 0.f, dmx = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            sx += x[s];
            sxl = fmaf(x[s], lam[s], sxl);
            rmax = fmaxf(rmax, fabsf(rd[s]));
            if (valid[s]) dmx = fmaxf(dmx, fminf(x[s], lam[s]));
        }
        rp = group_sum(sx, G) - 1.0f;
        mu = group_sum(sxl, G) * invP;
        rdmax = group_max(rmax, G);
        dec = group_max(dmx, G);
    };

    // All warps of a block iterate together (one block barrier per trip):
    // they then fetch the same instructions at about the same time, which
    // keeps the large unrolled loop body in the instruction cache.
    while (__syncthreads_or(alive)) {
        residual();

        // ---- leave the active set / refill (per group).  A group whose
        // pixel stopped stores it and takes the next one; the warp then
        // recomputes the residual (unchanged for the other groups) and all
        // groups take their Newton step in this same trip.  Each pass of the
        // refill loop consumes work items, so it ends.
        auto stop_test = [&]() -> bool {
            bool d;
            if (!ACC) d = (mu <= a.mu_ref) || (it >= a.max_iter);
            else d = ((rdmax <= a.tol_d) && (dec <= a.tol_c)) || (it >= a.max_iter);
            return d && alive;
        };
        bool done = stop_test();
        while (__any_sync(FULL, done)) {
            if (done) {
                const size_t base = (size_t)pix * P;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int i = s * G + t;
                    float *xo = BATCH ? cb->x_state : a.x_state, *lo = BATCH ? cb->lam_state : a.lam_state;
                    if (valid[s]) { xo[base + i] = x[s]; lo[base + i] = lam[s]; }
                }
                const bool conv = (rdmax <= a.tol_d) && (dec <= a.tol_c);
                if (t == 0) {
                    (BATCH ? cb->nu_state : a.nu_state)[pix] = nu;
                    if (!ACC) (BATCH ? cb->it_state : a.it_state)[pix] = it;
                    else {
                        a.it_state[pix] = conv ? it : -it;
                        if (!conv) atomicAdd(a.n_notconv, 1ULL);
                    }
                }
                pix = fetch();
                alive = has(pix);
                if (alive) load_pixel(pix);
            }
            residual();
            done = stop_test();
        }
        if (!__any_sync(FULL, alive)) continue;

        // ---- barrier Hessian H = G~ + diag(lambda / x), lower rows in registers
        float H[NS][PP];
        auto Dof = [&](int s) -> float { return valid[s] ? fminf(__fdividef(lam[s], x[s]), DMAX) : 1.f; };
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int i = s * G + t;
            const float Ds = Dof(s);
            const float *grow = gG + i * GST;
#pragma unroll
            for (int j4 = 0; j4 < (s + 1) * G / 4; ++j4) {
                const float4 g = ldG4(grow + 4 * j4);
                H[s][4 * j4 + 0] = g.x; H[s][4 * j4 + 1] = g.y;
                H[s][4 * j4 + 2] = g.z; H[s][4 * j4 + 3] = g.w;
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int j = s * G + q;
                if (!valid[s]) H[s][j] = (q == t) ? 1.f : 0.f;
                else if (q == t) H[s][j] += Ds;
            }
            if (!valid[s]) {
#pragma unroll
                for (int j = 0; j < s * G; ++j) H[s][j] = 0.f;
            }
        }

        // ---- factorise H = L L^T; eliminate rhs B1 = 1, B2 = r_aff = -r_d - lambda
        float B1[NS], B2[NS], dinv[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) { B1[s] = valid[s] ? 1.f : 0.f; B2[s] = -rd[s] - lam[s]; }
        const float *lb = colbuf + t;      // L[s*G + t][k] = lb[C::coloff(k) + s*G]
        auto inverse_blocks = [&]() {
            // ---- inverses M_b of the G x G diagonal blocks of L, written over the
            // blocks' strictly lower entries in the column buffer (the
            // factorisation is done with them); diag(M_b) = 1/L_kk stays in dinv
            // with the row's owner.  Lane t forms column t of M_b by forward
            // substitution; the block's entries are read by the whole group
            // (broadcast) before any lane writes.
    #pragma unroll
            for (int b = 0; b < NS; ++b) {
                float dq[G], m[G];
    #pragma unroll
                for (int q = 0; q < G; ++q) dq[q] = __shfl_sync(FULL, dinv[b], q, G);
    #pragma unroll
                for (int q = 0; q < G; ++q) {
                    float acc = 0.f;
    #pragma unroll
                    for (int r = 0; r < q; ++r) acc = fmaf(colbuf[C::coloff(b * G + r) + b * G + q], m[r], acc);
                    m[q] = (q == t) ? dinv[b] : ((q > t) ? -dq[q] * acc : 0.f);
                }
                __syncwarp();
                float *ct = colbuf + C::coloff(b * G + t) + b * G;
    #pragma unroll
                for (int q = 1; q < G; ++q)
                    if (q > t) ct[q] = m[q];
            }
            __syncwarp();
        };
        if constexpr (G == 4) {
            // Blocks of G = 4 columns (slot b).  (A) the group's four rows of
            // the diagonal block and their right-hand sides are exchanged
            // through shared memory; every lane factors the 4 x 4 block, solves
            // its right-hand sides and forms its inverse M_b (stored in the
            // block's strictly lower column slots for the triangular solves;
            // diag M_b = 1/L_kk stays in dinv).  (B) each lane forms its panel
            // rows L[i][4b..4b+3] = H[i][4b..4b+3] L_bb^-T in place (register
            // indices stay compile-time), stores them as columns and
            // eliminates its right-hand sides.  (C) rank-4 update of the later
            // blocks: per panel column one LDS.128 per four rows of the
            // trailing matrix, two packed FMAs per owned row.  The next slot's
            // columns are updated first and its rows exchanged at once, so
            // that the next block's factorisation (a short serial chain) can
            // overlap the rest of this update (lookahead).
            float *xrow = xbuf + 8 * t;
            float A[4][4], rb1[4], rb2[4];
            // exchange of the diagonal block rows of slot bb (after its
            // trailing updates) and their right-hand sides
            auto exchange = [&](auto bbc) {
                constexpr int bb = decltype(bbc)::value;
                *reinterpret_cast<float4 *>(xrow) = make_float4(H[bb][4 * bb], H[bb][4 * bb + 1], H[bb][4 * bb + 2], H[bb][4 * bb + 3]);
                *reinterpret_cast<float2 *>(xrow + 4) = make_float2(B1[bb], B2[bb]);
                __syncwarp();
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float4 rv = *reinterpret_cast<const float4 *>(xbuf + 8 * p);
                    const float2 bv = *reinterpret_cast<const float2 *>(xbuf + 8 * p + 4);
                    A[p][0] = rv.x; A[p][1] = rv.y; A[p][2] = rv.z; A[p][3] = rv.w;
                    rb1[p] = bv.x; rb2[p] = bv.y;
                }
            };
            exchange(std::integral_constant<int, 0>{});
            lm_static_for<NS>([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                float dq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float dd = A[q][q];
#pragma unroll
                    for (int r = 0; r < q; ++r) dd = fmaf(-A[q][r], A[q][r], dd);
                    dd = (dd > TINY) ? dd : BIGPIV;
                    const float rq = rsqrtf(dd);
                    dq[q] = rq;
#pragma unroll
                    for (int p = q + 1; p < 4; ++p) {
                        float v = A[p][q];
#pragma unroll
                        for (int r = 0; r < q; ++r) v = fmaf(-A[p][r], A[q][r], v);
                        A[p][q] = v * rq;
                    }
                }
                float z1[4], z2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float u1 = rb1[q], u2 = rb2[q];
#pragma unroll
                    for (int r = 0; r < q; ++r) { u1 = fmaf(-A[q][r], z1[r], u1); u2 = fmaf(-A[q][r], z2[r], u2); }
                    z1[q] = u1 * dq[q]; z2[q] = u2 * dq[q];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float mc[4];
                    mc[q] = dq[q];
#pragma unroll
                    for (int p = q + 1; p < 4; ++p) {
                        float v = 0.f;
#pragma unroll
                        for (int r = q; r < p; ++r) v = fmaf(A[p][r], mc[r], v);
                        mc[p] = -dq[p] * v;
                        colbuf[C::coloff(4 * b + q) + 4 * b + p] = mc[p];
                    }
                }
                dinv[b] = t == 0 ? dq[0] : t == 1 ? dq[1] : t == 2 ? dq[2] : dq[3];
                B1[b] = t == 0 ? z1[0] : t == 1 ? z1[1] : t == 2 ? z1[2] : z1[3];
                B2[b] = t == 0 ? z2[0] : t == 1 ? z2[1] : t == 2 ? z2[2] : z2[3];
#pragma unroll
                for (int s = b + 1; s < NS; ++s) {
                    float xq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float v = H[s][4 * b + q];
#pragma unroll
                        for (int r = 0; r < q; ++r) v = fmaf(-xq[r], A[q][r], v);
                        xq[q] = v * dq[q];
                        H[s][4 * b + q] = xq[q];
                        colbuf[t + C::coloff(4 * b + q) + 4 * s] = xq[q];
                        ffma2s(B1[s], B2[s], -xq[q], -xq[q], z1[q], z2[q], B1[s], B2[s]);
                    }
                }
                __syncwarp();
                // rank-4 update: first the next slot's columns (they feed the
                // next block's factorisation), then its exchange, then the
                // rest, which the scheduler can overlap with the next block
                auto update_cols = [&](int j4) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 lv = *reinterpret_cast<const float4 *>(colbuf + C::coloff(4 * b + q) + 4 * j4);
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            if (s < j4) continue;
                            const float nl = -H[s][4 * b + q];
                            ffma2s(H[s][4 * j4], H[s][4 * j4 + 1], nl, nl, lv.x, lv.y, H[s][4 * j4], H[s][4 * j4 + 1]);
                            ffma2s(H[s][4 * j4 + 2], H[s][4 * j4 + 3], nl, nl, lv.z, lv.w, H[s][4 * j4 + 2], H[s][4 * j4 + 3]);
                        }
                    }
                };
                if constexpr (b + 1 < NS) {
                    update_cols(b + 1);
                    exchange(std::integral_constant<int, b + 1>{});
#pragma unroll
                    for (int j4 = b + 2; j4 < NS; ++j4) update_cols(j4);
                }
            });
            __syncwarp();
        } else if constexpr (G == 8) {
            // Blocks of four columns inside slots of eight rows (two blocks
            // per slot): the same steps as for four-lane groups.  The rows of
            // block c are lanes t0..t0+3 (t0 = 4 (c % 2)) of slot c / 2; the
            // panel also takes the other half of that slot when c is even.
            // The strictly lower entries of L_bb go to the column slots; the
            // inverses of the 8 x 8 diagonal blocks are formed afterwards.
            constexpr int NB = PP / 4;
            float A[4][4], rb1[4], rb2[4];
            auto exchange = [&](auto ccc) {
                constexpr int cc = decltype(ccc)::value, sc = cc / 2, t0 = (cc % 2) * 4;
                if (t >= t0 && t < t0 + 4) {
                    float *xr = xbuf + 8 * (t - t0);
                    *reinterpret_cast<float4 *>(xr) = make_float4(H[sc][4 * cc], H[sc][4 * cc + 1], H[sc][4 * cc + 2], H[sc][4 * cc + 3]);
                    *reinterpret_cast<float2 *>(xr + 4) = make_float2(B1[sc], B2[sc]);
                }
                __syncwarp();
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const float4 rv = *reinterpret_cast<const float4 *>(xbuf + 8 * p);
                    const float2 bv = *reinterpret_cast<const float2 *>(xbuf + 8 * p + 4);
                    A[p][0] = rv.x; A[p][1] = rv.y; A[p][2] = rv.z; A[p][3] = rv.w;
                    rb1[p] = bv.x; rb2[p] = bv.y;
                }
            };
            exchange(std::integral_constant<int, 0>{});
            lm_static_for<NB>([&](auto ccc) {
                constexpr int c = decltype(ccc)::value, sc = c / 2, t0 = (c % 2) * 4;
                float dq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float dd = A[q][q];
#pragma unroll
                    for (int r = 0; r < q; ++r) dd = fmaf(-A[q][r], A[q][r], dd);
                    dd = (dd > TINY) ? dd : BIGPIV;
                    const float rq = rsqrtf(dd);
                    dq[q] = rq;
#pragma unroll
                    for (int p = q + 1; p < 4; ++p) {
                        float v = A[p][q];
#pragma unroll
                        for (int r = 0; r < q; ++r) v = fmaf(-A[p][r], A[q][r], v);
                        A[p][q] = v * rq;
                    }
                }
                float z1[4], z2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float u1 = rb1[q], u2 = rb2[q];
#pragma unroll
                    for (int r = 0; r < q; ++r) { u1 = fmaf(-A[q][r], z1[r], u1); u2 = fmaf(-A[q][r], z2[r], u2); }
                    z1[q] = u1 * dq[q]; z2[q] = u2 * dq[q];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int p = q + 1; p < 4; ++p) colbuf[C::coloff(4 * c + q) + 4 * c + p] = A[p][q];
                const int tr = t - t0;          // the lane's row in the block, if 0..3
                if (tr >= 0 && tr < 4) {
                    dinv[sc] = tr == 0 ? dq[0] : tr == 1 ? dq[1] : tr == 2 ? dq[2] : dq[3];
                    B1[sc] = tr == 0 ? z1[0] : tr == 1 ? z1[1] : tr == 2 ? z1[2] : z1[3];
                    B2[sc] = tr == 0 ? z2[0] : tr == 1 ? z2[1] : tr == 2 ? z2[2] : z2[3];
                }
#pragma unroll
                for (int s = sc; s < NS; ++s) {
                    // rows below the block: the later slots, and in slot sc
                    // (c even) the lanes of its second half
                    const bool row = s > sc || (t0 == 0 && t >= 4);
                    float xq[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float v = H[s][4 * c + q];
#pragma unroll
                        for (int r = 0; r < q; ++r) v = fmaf(-xq[r], A[q][r], v);
                        xq[q] = v * dq[q];
                    }
                    if (row) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            H[s][4 * c + q] = xq[q];
                            colbuf[t + C::coloff(4 * c + q) + 8 * s] = xq[q];
                            ffma2s(B1[s], B2[s], -xq[q], -xq[q], z1[q], z2[q], B1[s], B2[s]);
                        }
                    }
                }
                __syncwarp();
                // rank-4 update of the later column blocks (in slot sc, the
                // lanes above the panel update entries above the diagonal:
                // never read)
                auto update_cols = [&](int c2) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 lv = *reinterpret_cast<const float4 *>(colbuf + C::coloff(4 * c + q) + 4 * c2);
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            if (s < c2 / 2) continue;
                            const float nl = -H[s][4 * c + q];
                            ffma2s(H[s][4 * c2], H[s][4 * c2 + 1], nl, nl, lv.x, lv.y, H[s][4 * c2], H[s][4 * c2 + 1]);
                            ffma2s(H[s][4 * c2 + 2], H[s][4 * c2 + 3], nl, nl, lv.z, lv.w, H[s][4 * c2 + 2], H[s][4 * c2 + 3]);
                        }
                    }
                };
                if constexpr (c + 1 < NB) {
                    update_cols(c + 1);
                    exchange(std::integral_constant<int, c + 1>{});
#pragma unroll
                    for (int c2 = c + 2; c2 < NB; ++c2) update_cols(c2);
                }
            });
            __syncwarp();
            inverse_blocks();
        } else {
            // Column k = sk*G + tk: the slot block sk is unrolled (register
            // indices of H stay compile-time), the G columns of a block share one
            // copy of the code (rolled loop over tk, column picked by selects).
            // The loop body is then about 1/G of the fully unrolled one.
#pragma unroll
            for (int sk = 0; sk < NS; ++sk) {
#pragma unroll 1
                for (int tk = 0; tk < G; ++tk) {
                    const int k = sk * G + tk;
                    float hk[NS];
#pragma unroll
                    for (int s = sk; s < NS; ++s) {
                        float h = H[s][sk * G];
#pragma unroll
                        for (int q = 1; q < G; ++q) h = (tk == q) ? H[s][sk * G + q] : h;
                        hk[s] = h;
                    }
                    float d = __shfl_sync(FULL, hk[sk], tk, G);
                    d = (d > TINY) ? d : BIGPIV;
                    const float r = rsqrtf(d);
                    float *col = colbuf + C::colstart(k) - C::alignrow(k);
                    float lik[NS];
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        const bool below = (s > sk) || (s == sk && t > tk);
                        lik[s] = (s >= sk && below) ? hk[s] * r : 0.f;
                        if (s >= sk && below) col[s * G + t] = lik[s];
                    }
                    float z1 = 0.f, z2 = 0.f;
                    if (t == tk) {
                        dinv[sk] = r;                 // 1 / L_kk, kept by the row's owner
                        z1 = B1[sk] * r; z2 = B2[sk] * r;
                        B1[sk] = z1; B2[sk] = z2;
                    }
                    __syncwarp();
                    z1 = __shfl_sync(FULL, z1, tk, G);
                    z2 = __shfl_sync(FULL, z2, tk, G);
                    // columns of block sk right of k (runtime test j > k)
#pragma unroll
                    for (int j4 = sk * G / 4; j4 < (sk + 1) * G / 4; ++j4) {
                        const float4 lv = *reinterpret_cast<const float4 *>(col + 4 * j4);
                        const float lc[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int j = 4 * j4 + q;
                            if (j > k) {
#pragma unroll
                                for (int s = sk; s < NS; ++s) H[s][j] = fmaf(-lik[s], lc[q], H[s][j]);
                            }
                        }
                    }
                    // columns of the later blocks (the bulk of the update)
                    float nl[NS];
#pragma unroll
                    for (int s = sk; s < NS; ++s) nl[s] = -lik[s];
#pragma unroll
                    for (int j4 = (sk + 1) * G / 4; j4 < PP / 4; ++j4) {
                        const float4 lv = *reinterpret_cast<const float4 *>(col + 4 * j4);
#pragma unroll
                        for (int s = (4 * j4) / G; s < NS; ++s) {
                            ffma2s(H[s][4 * j4], H[s][4 * j4 + 1], nl[s], nl[s], lv.x, lv.y, H[s][4 * j4], H[s][4 * j4 + 1]);
                            ffma2s(H[s][4 * j4 + 2], H[s][4 * j4 + 3], nl[s], nl[s], lv.z, lv.w, H[s][4 * j4 + 2], H[s][4 * j4 + 3]);
                        }
                    }
#pragma unroll
                    for (int s = sk; s < NS; ++s) ffma2s(B1[s], B2[s], nl[s], nl[s], z1, z2, B1[s], B2[s]);
                }
            }
            __syncwarp();


            inverse_blocks();
        }

        // forward solve L z = v in place, by blocks of G rows: the block's G
        // values are gathered by shuffles, multiplied by M_b (row t), then
        // scattered into the later blocks (their columns of L read at
        // compile-time offsets, conflict-free)
        auto fwd_solve = [&](float (&v)[NS]) {
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                float y[G];
#pragma unroll
                for (int q = 0; q < G; ++q) y[q] = __shfl_sync(FULL, v[b], q, G);
                float z = dinv[b] * v[b];
#pragma unroll
                for (int q = 0; q < G - 1; ++q)
                    if (q < t) z = fmaf(lb[C::coloff(b * G + q) + b * G], y[q], z);
                v[b] = z;
                if (b + 1 < NS) {
                    float zq[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) zq[q] = __shfl_sync(FULL, z, q, G);
#pragma unroll
                    for (int s = b + 1; s < NS; ++s) {
#pragma unroll
                        for (int q = 0; q < G; ++q) v[s] = fmaf(-lb[C::coloff(b * G + q) + s * G], zq[q], v[s]);
                    }
                }
            }
        };
        // back solve L^T w = v in place, by blocks from the last: the dot
        // products of the block's columns with the solved rows below are
        // summed over the group (reduce-scatter: lane t receives column t's),
        // then the block is solved with M_b^T
        auto back_solve = [&](float (&v)[NS]) {
#pragma unroll
            for (int b = NS - 1; b >= 0; --b) {
                float d[G];
#pragma unroll
                for (int q = 0; q < G; ++q) {
                    float acc = 0.f;
#pragma unroll
                    for (int s = b + 1; s < NS; ++s) acc = fmaf(lb[C::coloff(b * G + q) + s * G], v[s], acc);
                    d[q] = acc;
                }
#pragma unroll
                for (int off = G / 2; off >= 1; off >>= 1) {
                    const bool hi = (t & off) != 0;
#pragma unroll
                    for (int i = 0; i < off; ++i) {
                        const float keep = hi ? d[i + off] : d[i];
                        const float send = hi ? d[i] : d[i + off];
                        d[i] = keep + __shfl_xor_sync(FULL, send, off);
                    }
                }
                const float yv = v[b] - d[0];
                float y[G];
#pragma unroll
                for (int q = 0; q < G; ++q) y[q] = __shfl_sync(FULL, yv, q, G);
                float w = dinv[b] * yv;
                const float *ct = colbuf + C::coloff(b * G + t) + b * G;
#pragma unroll
                for (int q = 1; q < G; ++q)
                    if (q > t) w = fmaf(ct[q], y[q], w);
                v[b] = w;
            }
        };

        // ---- predictor (affine scaling direction) and corrector.  The two
        // back solves share one copy of their (unrolled) code: a two-trip
        // loop kept rolled, which halves that part of the loop body and its
        // instruction-cache footprint.
        float p11 = 0.f, p1a = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) { p11 = fmaf(B1[s], B1[s], p11); p1a = fmaf(B1[s], B2[s], p1a); }
        const float a11 = group_sum(p11, G);
        const float a1a = group_sum(p1a, G);
        const float dnu_a = (a1a + rp) / a11;
        float dxa[NS], corr[NS], dnu_c = 0.f, ap = 1.f, ad = 1.f;
        float v[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) { v[s] = fmaf(-dnu_a, B1[s], B2[s]); corr[s] = 0.f; dxa[s] = 0.f; }
#pragma unroll 1
        for (int trip = 0; trip < 2; ++trip) {
            back_solve(v);
            if (trip == 1) break;
            // affine step: dlam_aff, step lengths, mu_aff, centering sigma
            float dla[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                dxa[s] = v[s];
                dla[s] = valid[s] ? fmaf(-Dof(s), dxa[s], -lam[s]) : 0.f;
                if (valid[s] && dxa[s] < 0.f) ap = fminf(ap, __fdividef(-x[s], dxa[s]));
                if (valid[s] && dla[s] < 0.f) ad = fminf(ad, __fdividef(-lam[s], dla[s]));
            }
            ap = group_min(ap, G);
            ad = group_min(ad, G);
            float pma = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) pma = fmaf(fmaf(ap, dxa[s], x[s]), fmaf(ad, dla[s], lam[s]), pma);
            const float mua = group_sum(pma, G) * invP;
            float sig = (mu > 0.f) ? mua / mu : 0.f;
            sig = fminf(sig * sig * sig, 1.f);
            const float smu = sig * mu;
            // corrector right-hand side -X^-1 (dx_aff o dlam_aff - sigma mu 1)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                corr[s] = valid[s] ? __fdividef(fmaf(dxa[s], dla[s], -smu), x[s]) : 0.f;
                v[s] = -corr[s];
            }
            fwd_solve(v);
            float p1c = 0.f;
#pragma unroll
            for (int s = 0; s < NS; ++s) p1c = fmaf(B1[s], v[s], p1c);
            dnu_c = group_sum(p1c, G) / a11;
#pragma unroll
            for (int s = 0; s < NS; ++s) v[s] = fmaf(-dnu_c, B1[s], v[s]);
        }

        float dx[NS], dl[NS];
        ap = 1.f; ad = 1.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            dx[s] = dxa[s] + v[s];
            dl[s] = valid[s] ? fmaf(-Dof(s), dx[s], -lam[s] - corr[s]) : 0.f;
            if (valid[s] && dx[s] < 0.f) ap = fminf(ap, __fdividef(-x[s], dx[s]));
            if (valid[s] && dl[s] < 0.f) ad = fminf(ad, __fdividef(-lam[s], dl[s]));
        }
        ap = group_min(ap, G);
        ad = group_min(ad, G);
        const float alpha = fminf(1.f, a.eta * fminf(ap, ad));
        const float dnu = dnu_a + dnu_c;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (valid[s]) {
                x[s] = fmaxf(fmaf(alpha, dx[s], x[s]), TINY);
                lam[s] = fmaxf(fmaf(alpha, dl[s], lam[s]), TINY);
            }
        }
        nu = fmaf(alpha, dnu, nu);
        ++it;
    }
}

}  // namespace lm
