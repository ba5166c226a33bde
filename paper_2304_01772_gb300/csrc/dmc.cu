// dmc.cu -- differentiable Monte Carlo (Alg. 2 of Farias et al., arXiv
// 2304.01772, Sec. "Methods"): relaxed checkerboard sweeps of Ising lattices
// with one exchange parameter per bond, their reverse pass, the L2 pattern
// loss and the discretisation of Sec. "Optimization of the exchange
// parameters".
//
// Sub-step of colour c, every site i with (x + y) & 1 == c at once:
//   n = sum_j J_ij s_j,  dE = 2 s (n + h)  (proposal s' = -s under
//   H = -sum J_ij s_i s_j - h sum s_i),  p = exp(-beta dE) (not clipped),
//   r = (u >> 8) 2^-24 (u: the site's Philox lane, Ising layout: counter
//   (k >> 2, lattice, sweep, c), lane k & 3, k = (y L + x) >> 1),
//   q = 1 / (1 + exp(-alpha (p - r))),  s <- q s' + (1 - q) s.
// Reverse pass, with w_i = dL/ds_new(i) * 4 alpha beta p q (1 - q) s_i^2:
//   dL/ds_old(i) = dL/ds_new(i) ((1 - 2q) + 4 alpha beta p q (1 - q) s_i (n_i + h)),
//   dL/ds_old(j) = dL/ds_new(j) + sum_i w_i J_ij  (j passive),
//   dL/dJ_ij += w_i s_j.
//
// One block per lattice; the lattice (L <= 64, L % 8 == 0) lives in shared
// memory for all sub-steps.  The forward pass records only the old values of
// each sub-step's active sites (the passive ones do not change), so the tape
// costs 2 B per site and sub-step; the reverse pass restores them in turn.
// Each bond has exactly one passive end per sub-step, whose thread updates
// its gradient: no atomics.  Arithmetic is float32 as in the paper's PyTorch
// form; expf is CUDA's.
#include "internal.h"

namespace spinmc {

namespace {

constexpr int kDmcThreads = 256;

struct DmcGeom {
    int L, half, N;   // side, L / 2, L * L
};

__device__ __forceinline__ float dmc_uniform(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

// Weighted neighbour sum of site i = (x, y).
__device__ __forceinline__ float dmc_field(const DmcGeom &g, const float *s, const float *Jr,
                                           const float *Jd, int i, int x, int y) {
    const int xl = x == 0 ? g.L - 1 : x - 1, xr = x == g.L - 1 ? 0 : x + 1;
    const int yu = y == 0 ? g.L - 1 : y - 1, yd = y == g.L - 1 ? 0 : y + 1;
    return Jr[i] * s[y * g.L + xr] + Jr[y * g.L + xl] * s[y * g.L + xl] + Jd[i] * s[yd * g.L + x] +
           Jd[yu * g.L + x] * s[yu * g.L + x];
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void load_f4(float *dst, const float *src, int n) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int v = threadIdx.x; v < n / 4; v += blockDim.x) d4[v] = s4[v];
}

__device__ __forceinline__ void store_f4(float *dst, const float *src, int n) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int v = threadIdx.x; v < n / 4; v += blockDim.x) d4[v] = s4[v];
}

// Forward sub-step `sub` of lattice `lat` on the block's shared copy; the
// active sites' old values go to tape (N / 2 floats, compressed order; shared
// or global memory).  Ends with a block barrier.
__device__ __forceinline__ void dmc_forward_substep(const DmcGeom &g, float *s, const float *Jr, const float *Jd,
                                                    float *tape, int lat, uint32_t sweep, int c, float beta,
                                                    float h, float alpha, uint32_t k0, uint32_t k1) {
    const int gpr = g.half / 4;   // Philox groups per row: a group's four sites share a row
    for (int grp = threadIdx.x; grp < g.N / 8; grp += blockDim.x) {
        const uint4 r4 = philox4x32_10(make_uint4((uint32_t)grp, (uint32_t)lat, sweep, (uint32_t)c), k0, k1);
        const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
        const int y = grp / gpr, x0 = 8 * (grp - y * gpr) + ((y + c) & 1);
        float old[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int x = x0 + 2 * l, i = y * g.L + x;
            const float si = s[i];
            const float n = dmc_field(g, s, Jr, Jd, i, x, y);
            const float p = expf(-beta * (2.0f * si * (n + h)));
            const float q = __frcp_rn(1.0f + expf(-alpha * (p - dmc_uniform(rr[l]))));
            old[l] = si;
            s[i] = q * (-si) + (1.0f - q) * si;
        }
        reinterpret_cast<float4 *>(tape)[grp] = make_float4(old[0], old[1], old[2], old[3]);
    }
    __syncthreads();
}

// Reverse of sub-step `sub`: s holds the state after it and becomes the state
// before it; gs likewise for the adjoint; gJr / gJd accumulate.  w: N / 2
// floats of scratch; it may be the sub-step's own tape slot (each thread reads
// its four old values before it writes their four w).  Ends with a block
// barrier.
template <bool GJ = true>
__device__ __forceinline__ void dmc_backward_substep(const DmcGeom &g, float *s, float *gs, const float *Jr,
                                                     const float *Jd, float *gJr, float *gJd, float *w,
                                                     const float *tape, int lat, uint32_t sweep, int c,
                                                     float beta, float h, float alpha, uint32_t k0,
                                                     uint32_t k1) {
    const float c4 = 4.0f * alpha * beta;
    // active sites: restore the old value, form w and the direct term
    const int gpr = g.half / 4;
    for (int grp = threadIdx.x; grp < g.N / 8; grp += blockDim.x) {
        const uint4 r4 = philox4x32_10(make_uint4((uint32_t)grp, (uint32_t)lat, sweep, (uint32_t)c), k0, k1);
        const uint32_t rr[4] = {r4.x, r4.y, r4.z, r4.w};
        const float4 o4 = reinterpret_cast<const float4 *>(tape)[grp];
        const float old[4] = {o4.x, o4.y, o4.z, o4.w};
        const int y = grp / gpr, x0 = 8 * (grp - y * gpr) + ((y + c) & 1);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int x = x0 + 2 * l, i = y * g.L + x;
            const float si = old[l];
            const float n = dmc_field(g, s, Jr, Jd, i, x, y);
            const float p = expf(-beta * (2.0f * si * (n + h)));
            const float q = __frcp_rn(1.0f + expf(-alpha * (p - dmc_uniform(rr[l]))));
            const float common = c4 * p * q * (1.0f - q);
            const float gi = gs[i];
            w[4 * grp + l] = gi * common * si * si;
            gs[i] = gi * ((1.0f - 2.0f * q) + common * si * (n + h));
            s[i] = si;
        }
    }
    __syncthreads();
    // passive sites: their adjoint gains sum_i w_i J_ij; their four bonds gain w_i s_j
    for (int k = threadIdx.x; k < g.N / 2; k += blockDim.x) {
        const int y = k / g.half, x = 2 * (k - y * g.half) + ((y + c + 1) & 1), j = y * g.L + x;
        const int xl = x == 0 ? g.L - 1 : x - 1, xr = x == g.L - 1 ? 0 : x + 1;
        const int yu = y == 0 ? g.L - 1 : y - 1, yd = y == g.L - 1 ? 0 : y + 1;
        const int iL = y * g.L + xl, iR = y * g.L + xr, iU = yu * g.L + x, iD = yd * g.L + x;
        const float wl = w[iL >> 1], wr = w[iR >> 1], wu = w[iU >> 1], wd = w[iD >> 1];
        const float sj = s[j];
        gs[j] += wr * Jr[j] + wl * Jr[iL] + wd * Jd[j] + wu * Jd[iU];
        if (GJ) {
            gJr[j] += wr * sj;
            gJr[iL] += wl * sj;
            gJd[j] += wd * sj;
            gJd[iU] += wu * sj;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDmcThreads) dmc_forward_kernel(DmcArgs a) {
    extern __shared__ __align__(16) float sm[];
    const DmcGeom g{a.L, a.L / 2, a.L * a.L};
    float *s = sm, *Jr = sm + g.N, *Jd = sm + 2 * g.N;
    const int n_sub = 2 * a.n_sweeps;
    for (int lat = blockIdx.x; lat < a.n_lat; lat += gridDim.x) {
        load_f4(s, a.spins + (size_t)lat * g.N, g.N);
        load_f4(Jr, a.J + (size_t)lat * 2 * g.N, g.N);
        load_f4(Jd, a.J + (size_t)lat * 2 * g.N + g.N, g.N);
        __syncthreads();
        float *tape = a.tape + (size_t)lat * n_sub * (g.N / 2);
        for (int sub = 0; sub < n_sub; ++sub)
            dmc_forward_substep(g, s, Jr, Jd, tape + (size_t)sub * (g.N / 2), lat,
                                a.first_sweep + (uint32_t)(sub >> 1), sub & 1, a.beta, a.h, a.alpha, a.k0, a.k1);
        store_f4(a.spins + (size_t)lat * g.N, s, g.N);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kDmcThreads) dmc_backward_kernel(DmcArgs a) {
    extern __shared__ __align__(16) float sm[];
    const DmcGeom g{a.L, a.L / 2, a.L * a.L};
    float *s = sm, *gs = sm + g.N, *Jr = sm + 2 * g.N, *Jd = sm + 3 * g.N;
    float *gJr = sm + 4 * g.N, *gJd = sm + 5 * g.N, *w = sm + 6 * g.N;   // w: N / 2
    const int n_sub = 2 * a.n_sweeps;
    for (int lat = blockIdx.x; lat < a.n_lat; lat += gridDim.x) {
        load_f4(s, a.spins + (size_t)lat * g.N, g.N);
        load_f4(gs, a.grad_spins + (size_t)lat * g.N, g.N);
        load_f4(Jr, a.J + (size_t)lat * 2 * g.N, g.N);
        load_f4(Jd, a.J + (size_t)lat * 2 * g.N + g.N, g.N);
        for (int i = threadIdx.x; i < g.N; i += blockDim.x) gJr[i] = gJd[i] = 0.0f;
        __syncthreads();
        const float *tape = a.tape + (size_t)lat * n_sub * (g.N / 2);
        for (int sub = n_sub - 1; sub >= 0; --sub)
            dmc_backward_substep(g, s, gs, Jr, Jd, gJr, gJd, w, tape + (size_t)sub * (g.N / 2), lat,
                                 a.first_sweep + (uint32_t)(sub >> 1), sub & 1, a.beta, a.h, a.alpha, a.k0, a.k1);
        store_f4(a.grad_spins + (size_t)lat * g.N, gs, g.N);
        store_f4(a.grad_J + (size_t)lat * 2 * g.N, gJr, g.N);
        store_f4(a.grad_J + (size_t)lat * 2 * g.N + g.N, gJd, g.N);
        __syncthreads();
    }
}

// One whole optimisation iteration per lattice with everything in shared
// memory: forward sweeps (tape kept on chip), loss and its gradient, reverse
// pass, Adam on the couplings, and the discretised state written back.  HBM
// traffic per site: spins and target in, spins out, couplings and both Adam
// moments in and out.
constexpr int kDmcStepThreads = 512;

__global__ void __launch_bounds__(kDmcStepThreads, 2) dmc_step_kernel(DmcStepArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[kDmcStepThreads / 32];
    const DmcGeom g{a.L, a.L / 2, a.L * a.L};
    float *s = sm, *gs = sm + g.N, *Jr = sm + 2 * g.N, *Jd = sm + 3 * g.N;
    float *gJr = sm + 4 * g.N, *gJd = sm + 5 * g.N;
    float *tape = sm + 6 * g.N;   // 2 n_sweeps x N / 2; the reverse pass reuses each slot for its w
    const int n_sub = 2 * a.n_sweeps;
    for (int lat = blockIdx.x; lat < a.n_lat; lat += gridDim.x) {
        float *spins = a.spins + (size_t)lat * g.N;
        float *J = a.J + (size_t)lat * 2 * g.N;
        // pull this block's next lattice into L2 while this one is computed
        const int nxt = lat + gridDim.x;
        if (nxt < a.n_lat) {
            const size_t o1 = (size_t)nxt * g.N, o2 = (size_t)nxt * 2 * g.N;
            for (int line = threadIdx.x; line < g.N / 32; line += blockDim.x) {   // 128-byte lines
                prefetch_l2(a.spins + o1 + 32 * line);
                prefetch_l2(a.target + o1 + 32 * line);
            }
            for (int line = threadIdx.x; line < g.N / 16; line += blockDim.x) {
                prefetch_l2(a.J + o2 + 32 * line);
                prefetch_l2(a.m + o2 + 32 * line);
                prefetch_l2(a.v + o2 + 32 * line);
            }
        }
        load_f4(s, spins, g.N);
        load_f4(Jr, J, g.N);
        load_f4(Jd, J + g.N, g.N);
        __syncthreads();
        for (int sub = 0; sub < n_sub; ++sub)
            dmc_forward_substep(g, s, Jr, Jd, tape + (size_t)sub * (g.N / 2), lat,
                                a.first_sweep + (uint32_t)(sub >> 1), sub & 1, a.beta, a.h, a.alpha, a.k0, a.k1);
        // loss of the relaxed state, its gradient, and the discretised state
        const float4 *t4 = reinterpret_cast<const float4 *>(a.target + (size_t)lat * g.N);
        double acc = 0.0;
        for (int i4 = threadIdx.x; i4 < g.N / 4; i4 += blockDim.x) {
            const float4 tt = t4[i4];
            const float4 ss = reinterpret_cast<const float4 *>(s)[i4];
            const float d[4] = {tt.x - ss.x, tt.y - ss.y, tt.z - ss.z, tt.w - ss.w};
            const float sv[4] = {ss.x, ss.y, ss.z, ss.w};
#pragma unroll
            for (int l = 0; l < 4; ++l) acc += (double)d[l] * (double)d[l];
            reinterpret_cast<float4 *>(gs)[i4] = make_float4(-2.0f * d[0], -2.0f * d[1], -2.0f * d[2], -2.0f * d[3]);
            reinterpret_cast<float4 *>(spins)[i4] =
                make_float4(sv[0] < 0.0f ? -1.0f : 1.0f, sv[1] < 0.0f ? -1.0f : 1.0f, sv[2] < 0.0f ? -1.0f : 1.0f,
                            sv[3] < 0.0f ? -1.0f : 1.0f);
            reinterpret_cast<float4 *>(gJr)[i4] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4 *>(gJd)[i4] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kDmcStepThreads / 32; ++k) t += red[k];
            a.loss[lat] = t;
        }
        for (int sub = n_sub - 1; sub >= 0; --sub) {
            float *slot = tape + (size_t)sub * (g.N / 2);
            dmc_backward_substep(g, s, gs, Jr, Jd, gJr, gJd, slot, slot, lat, a.first_sweep + (uint32_t)(sub >> 1),
                                 sub & 1, a.beta, a.h, a.alpha, a.k0, a.k1);
        }
        // Adam on the 2N couplings of this lattice
        // (Jr, Jd and gJr, gJd are adjacent in shared memory: bond b < 2N is Jr[b])
        float4 *m4 = reinterpret_cast<float4 *>(a.m + (size_t)lat * 2 * g.N);
        float4 *v4 = reinterpret_cast<float4 *>(a.v + (size_t)lat * 2 * g.N);
        float4 *J4 = reinterpret_cast<float4 *>(J);
        const float4 *P4 = reinterpret_cast<const float4 *>(Jr), *G4 = reinterpret_cast<const float4 *>(gJr);
        for (int b = threadIdx.x; b < g.N / 2; b += blockDim.x) {
            float4 p = P4[b], mm = m4[b], vv = v4[b];
            const float4 gg = G4[b];
            adam_element(p.x, mm.x, vv.x, gg.x, a.lr, a.b1, a.b2, a.eps, a.c1, a.c2);
            adam_element(p.y, mm.y, vv.y, gg.y, a.lr, a.b1, a.b2, a.eps, a.c1, a.c2);
            adam_element(p.z, mm.z, vv.z, gg.z, a.lr, a.b1, a.b2, a.eps, a.c1, a.c2);
            adam_element(p.w, mm.w, vv.w, gg.w, a.lr, a.b1, a.b2, a.eps, a.c1, a.c2);
            m4[b] = mm;
            v4[b] = vv;
            J4[b] = p;
        }
        __syncthreads();
    }
}

// One iteration of the spin-value optimisation by differentiable Monte Carlo
// per lattice, in shared memory: relaxed sweeps F from the spins s, the energy
// gradient of F(s), the reverse pass to dE(F(s))/ds (no coupling gradients),
// then s <- discretise(clip(s - eta sign(.), -1, 1)); energy[lat] = E of
// discretise(F(s)), the state the simulation produced.
__global__ void __launch_bounds__(kDmcStepThreads, 2) dmc_spin_iter_kernel(DmcSpinIterArgs a) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[kDmcStepThreads / 32];
    const DmcGeom g{a.L, a.L / 2, a.L * a.L};
    float *s0 = sm, *s = sm + g.N, *gs = sm + 2 * g.N, *Jr = sm + 3 * g.N, *Jd = sm + 4 * g.N;
    float *tape = sm + 5 * g.N;   // 2 n_sweeps x N / 2; the reverse pass reuses each slot for its w
    const int n_sub = 2 * a.n_sweeps;
    for (int lat = blockIdx.x; lat < a.n_lat; lat += gridDim.x) {
        float *spins = a.spins + (size_t)lat * g.N;
        const float *J = a.J + (size_t)lat * 2 * g.N;
        load_f4(s0, spins, g.N);
        load_f4(s, spins, g.N);
        load_f4(Jr, J, g.N);
        load_f4(Jd, J + g.N, g.N);
        __syncthreads();
        for (int sub = 0; sub < n_sub; ++sub)
            dmc_forward_substep(g, s, Jr, Jd, tape + (size_t)sub * (g.N / 2), lat,
                                a.first_sweep + (uint32_t)(sub >> 1), sub & 1, a.beta, a.h, a.alpha, a.k0, a.k1);
        // dE/ds of the relaxed state, and the energy of its discretisation
        double acc = 0.0;
        for (int i = threadIdx.x; i < g.N; i += blockDim.x) {
            const int y = i / g.L, x = i - y * g.L;
            gs[i] = -(dmc_field(g, s, Jr, Jd, i, x, y) + a.h);
            const int xr = x == g.L - 1 ? 0 : x + 1, yd = y == g.L - 1 ? 0 : y + 1;
            const double di = s[i] < 0.0f ? -1.0 : 1.0;
            const double dr = s[y * g.L + xr] < 0.0f ? -1.0 : 1.0, dd = s[yd * g.L + x] < 0.0f ? -1.0 : 1.0;
            acc -= (double)Jr[i] * di * dr + (double)Jd[i] * di * dd + (double)a.h * di;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kDmcStepThreads / 32; ++k) t += red[k];
            a.energy[lat] = t;
        }
        for (int sub = n_sub - 1; sub >= 0; --sub) {
            float *slot = tape + (size_t)sub * (g.N / 2);
            dmc_backward_substep<false>(g, s, gs, Jr, Jd, nullptr, nullptr, slot, slot, lat,
                                        a.first_sweep + (uint32_t)(sub >> 1), sub & 1, a.beta, a.h, a.alpha,
                                        a.k0, a.k1);
        }
        // quantised step on the start spins, then discretisation
        for (int i = threadIdx.x; i < g.N; i += blockDim.x) {
            const float gi = gs[i];
            const float v = s0[i] - a.eta * (gi > 0.0f ? 1.0f : (gi < 0.0f ? -1.0f : 0.0f));
            const float c = fminf(1.0f, fmaxf(-1.0f, v));
            spins[i] = c < 0.0f ? -1.0f : 1.0f;
        }
        __syncthreads();
    }
}

// loss[lat] = sum (target - s)^2 (double); grad = -2 (target - s).
__global__ void __launch_bounds__(kDmcThreads) dmc_loss_kernel(int n_lat, int N, const float *spins,
                                                               const float *target, float *grad,
                                                               double *loss) {
    __shared__ double red[kDmcThreads / 32];
    for (int lat = blockIdx.x; lat < n_lat; lat += gridDim.x) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const size_t o = (size_t)lat * N + i;
            const float d = target[o] - spins[o];
            acc += (double)d * (double)d;
            grad[o] = -2.0f * d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kDmcThreads / 32; ++k) t += red[k];
            loss[lat] = t;
        }
        __syncthreads();
    }
}

// energy[lat] = -sum_<ij> J_ij s_i s_j - h sum s_i (double); grad = -(n + h).
__global__ void __launch_bounds__(kDmcThreads) dmc_energy_kernel(int n_lat, int L, const float *J,
                                                                 const float *spins, float h, float *grad,
                                                                 double *energy) {
    __shared__ double red[kDmcThreads / 32];
    const DmcGeom g{L, L / 2, L * L};
    for (int lat = blockIdx.x; lat < n_lat; lat += gridDim.x) {
        const float *s = spins + (size_t)lat * g.N;
        const float *Jr = J + (size_t)lat * 2 * g.N, *Jd = Jr + g.N;
        double acc = 0.0;
        for (int i = threadIdx.x; i < g.N; i += blockDim.x) {
            const int y = i / L, x = i - y * L;
            const int xr = x == L - 1 ? 0 : x + 1, yd = y == L - 1 ? 0 : y + 1;
            const double si = s[i];
            acc -= (double)Jr[i] * si * (double)s[y * L + xr] + (double)Jd[i] * si * (double)s[yd * L + x] +
                   (double)h * si;
            if (grad) grad[(size_t)lat * g.N + i] = -(dmc_field(g, s, Jr, Jd, i, x, y) + h);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kDmcThreads / 32; ++k) t += red[k];
            energy[lat] = t;
        }
        __syncthreads();
    }
}

// s <- clip(s - eta sign(g), -1, 1), sign(0) = 0.
__global__ void dmc_spin_step_kernel(int64_t n, float *s, const float *g, float eta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float v = s[i] - eta * (gi > 0.0f ? 1.0f : (gi < 0.0f ? -1.0f : 0.0f));
        s[i] = fminf(1.0f, fmaxf(-1.0f, v));
    }
}

__global__ void dmc_discretize_kernel(int64_t n, float *s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s[i] = s[i] < 0.0f ? -1.0f : 1.0f;
}

int dmc_grid(int n_lat, int per_sm) { return n_lat < 152 * per_sm ? n_lat : 152 * per_sm; }

}  // namespace

size_t dmc_forward_smem(int L) { return sizeof(float) * 3 * (size_t)L * L; }
size_t dmc_backward_smem(int L) { return sizeof(float) * (6 * (size_t)L * L + (size_t)L * L / 2); }

cudaError_t launch_dmc_forward(const DmcArgs &a, cudaStream_t s) {
    const size_t sm = dmc_forward_smem(a.L);
    cudaError_t e = cudaFuncSetAttribute(dmc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    dmc_forward_kernel<<<dmc_grid(a.n_lat, 4), kDmcThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dmc_backward(const DmcArgs &a, cudaStream_t s) {
    const size_t sm = dmc_backward_smem(a.L);
    cudaError_t e = cudaFuncSetAttribute(dmc_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    dmc_backward_kernel<<<dmc_grid(a.n_lat, 2), kDmcThreads, sm, s>>>(a);
    return cudaGetLastError();
}

size_t dmc_step_smem(int L, int n_sweeps) {
    const size_t N = (size_t)L * L;
    return sizeof(float) * (6 * N + (size_t)n_sweeps * N);
}

cudaError_t launch_dmc_step(const DmcStepArgs &a, cudaStream_t s) {
    const size_t sm = dmc_step_smem(a.L, a.n_sweeps);
    cudaError_t e = cudaFuncSetAttribute(dmc_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    dmc_step_kernel<<<dmc_grid(a.n_lat, 2), kDmcStepThreads, sm, s>>>(a);
    return cudaGetLastError();
}

size_t dmc_spin_iter_smem(int L, int n_sweeps) {
    const size_t N = (size_t)L * L;
    return sizeof(float) * (5 * N + (size_t)n_sweeps * N);
}

cudaError_t launch_dmc_spin_iter(const DmcSpinIterArgs &a, cudaStream_t s) {
    const size_t sm = dmc_spin_iter_smem(a.L, a.n_sweeps);
    cudaError_t e = cudaFuncSetAttribute(dmc_spin_iter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    dmc_spin_iter_kernel<<<dmc_grid(a.n_lat, 2), kDmcStepThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dmc_loss(int n_lat, int N, const float *spins, const float *target, float *grad,
                            double *loss, cudaStream_t s) {
    dmc_loss_kernel<<<dmc_grid(n_lat, 8), kDmcThreads, 0, s>>>(n_lat, N, spins, target, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_dmc_energy(int n_lat, int L, const float *J, const float *spins, float h, float *grad,
                              double *energy, cudaStream_t s) {
    dmc_energy_kernel<<<dmc_grid(n_lat, 8), kDmcThreads, 0, s>>>(n_lat, L, J, spins, h, grad, energy);
    return cudaGetLastError();
}

cudaError_t launch_dmc_spin_step(int64_t n, float *spins, const float *grad, float eta, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    dmc_spin_step_kernel<<<blocks, 256, 0, s>>>(n, spins, grad, eta);
    return cudaGetLastError();
}

cudaError_t launch_dmc_discretize(int64_t n, float *spins, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    dmc_discretize_kernel<<<blocks, 256, 0, s>>>(n, spins);
    return cudaGetLastError();
}

}  // namespace spinmc
