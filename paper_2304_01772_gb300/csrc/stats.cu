// stats.cu -- observables and the fluctuation-estimator gradient.
//
// Per-sweep statistics are exact integers (Ising M, B; Potts B_eq, n_k; CPM
// contact counts C_ab and area sums V2, V1).  The sweep kernels accumulate
// their changes in `delta`; launch_finalize folds them into `cur` and writes
// a record.  The adjoint reduction forms exact moments sum X_i and
// sum X_i X_j in 128-bit integers; the finaliser turns them into
// d<O>/dtheta = <dO/dtheta> - beta Cov(O, dH/dtheta) in FP64.
#include "internal.h"

namespace spinmc {

namespace {

__device__ __forceinline__ int pair_idx(int a, int b, int n) {
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * n - lo * (lo - 1) / 2 + (hi - lo);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ void atomic_add_i64(int64_t *p, long long v) {
    if (v) atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}

// Ising / Potts statistics recomputed from the lattice (right and down bonds).
__global__ void stats_state_kernel(const void *spins, int model, const LatDev *lats, int width,
                                   int64_t *out) {
    __shared__ int shist[256];
    __shared__ long long r0[32], r1[32], r2[32];
    const int lat = blockIdx.y;
    const LatDev ld = lats[lat];
    const int L = ld.L;
    for (int k = threadIdx.x; k < 256; k += blockDim.x) shist[k] = 0;
    __syncthreads();
    long long a0 = 0, a1 = 0, a2 = 0;
    if (model == 0 && ld.fast && ld.geom == 0) {
        // +-1 bytes (0x01 / 0xFF): bit 7 marks -1, and bit 7 of a ^ b marks a
        // neighbour pair of opposite spins.  16 sites per thread: M = N - 2 n_down,
        // B = 2N - 2 n_unequal (right and down bonds).
        const uint4 *S4 = reinterpret_cast<const uint4 *>(static_cast<const int8_t *>(spins) + ld.offset);
        const int Lv = L >> 4;
        long long down = 0, uneq = 0;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < L * Lv; v += gridDim.x * blockDim.x) {
            const int y = v / Lv, j = v - y * Lv;
            const uint4 C = S4[v];
            const uint4 D = S4[(y == L - 1 ? 0 : y + 1) * Lv + j];
            const uint32_t nx = reinterpret_cast<const uint32_t *>(S4 + y * Lv + (j == Lv - 1 ? 0 : j + 1))[0];
            const uint32_t w[5] = {C.x, C.y, C.z, C.w, nx};
            const uint32_t d[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t r = __funnelshift_r(w[q], w[q + 1], 8);   // right neighbours
                down += __popc(w[q] & 0x80808080u);
                uneq += __popc((w[q] ^ r) & 0x80808080u) + __popc((w[q] ^ d[q]) & 0x80808080u);
            }
        }
        const long long n_site = 16ll * ((L * Lv - 1 - (blockIdx.x * blockDim.x + threadIdx.x)) /
                                         (gridDim.x * blockDim.x) + 1);
        const bool any = (int)(blockIdx.x * blockDim.x + threadIdx.x) < L * Lv;
        a0 = any ? n_site - 2 * down : 0;
        a1 = any ? 2 * n_site - 2 * uneq : 0;
    } else
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L, x = i - y * L;
        const int ir = y * L + (x == L - 1 ? 0 : x + 1);
        const int id = (y == L - 1 ? 0 : y + 1) * L + x;
        if (model == 0) {
            const int8_t *S = static_cast<const int8_t *>(spins) + ld.offset;
            const int s = S[i];
            a0 += s;
            a1 += s * (S[ir] + S[id]);
            if (ld.geom == 1)   // triangular: the third bond direction (x - 1, y + 1)
                a1 += s * S[(y == L - 1 ? 0 : y + 1) * L + (x == 0 ? L - 1 : x - 1)];
            if (ld.geom == 2) {   // diagonal bonds through (x + 1, y + 1) and (x + 1, y - 1)
                const int xr = x == L - 1 ? 0 : x + 1;
                a2 += s * (S[(y == L - 1 ? 0 : y + 1) * L + xr] + S[(y == 0 ? L - 1 : y - 1) * L + xr]);
            }
        } else {
            const uint8_t *S = static_cast<const uint8_t *>(spins) + ld.offset;
            const int s = S[i];
            a0 += (s == S[ir]) + (s == S[id]);
            atomicAdd(shist + s, 1);
        }
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if ((threadIdx.x & 31) == 0) {
        r0[threadIdx.x >> 5] = a0;
        r1[threadIdx.x >> 5] = a1;
        r2[threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    int64_t *o = out + (size_t)width * lat;
    if (threadIdx.x == 0) {
        long long s0 = 0, s1 = 0, s2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s0 += r0[w];
            s1 += r1[w];
            s2 += r2[w];
        }
        if (model == 0) {
            atomic_add_i64(o, s0);
            atomic_add_i64(o + 1, s1);
            if (width > 2) atomic_add_i64(o + 2, s2);
        } else {
            atomic_add_i64(o, s0);
        }
    }
    if (model == 1)
        for (int k = threadIdx.x; k < ld.q && k + 1 < width; k += blockDim.x)
            atomic_add_i64(o + 1 + k, shist[k]);
}

// CPM contacts (right, down-left, down, down-right: each unordered Moore pair once).
__global__ void stats_cpm_kernel(const int32_t *ids, int L, const uint8_t *type, int nt,
                                 const int32_t *vol, int n_cells, int target, int width,
                                 int64_t *out) {
    __shared__ int scnt[36];
    __shared__ long long r2[32], r1[32];
    for (int k = threadIdx.x; k < 36; k += blockDim.x) scnt[k] = 0;
    __syncthreads();
    const int hx[4] = {1, -1, 0, 1}, hy[4] = {0, 1, 1, 1};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L * L; i += gridDim.x * blockDim.x) {
        const int y = i / L, x = i - y * L;
        const int a = ids[i];
        if ((unsigned)a > (unsigned)n_cells) continue;
        for (int k = 0; k < 4; ++k) {
            int yy = y + hy[k], xx = x + hx[k];
            yy = yy >= L ? yy - L : yy;
            xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
            const int b = ids[yy * L + xx];
            if ((unsigned)b > (unsigned)n_cells) continue;
            if (a != b) atomicAdd(scnt + pair_idx(type[a], type[b], nt), 1);
        }
    }
    long long v2 = 0, v1 = 0;
    if (blockIdx.x == 0) {
        for (int c = 1 + threadIdx.x; c <= n_cells; c += blockDim.x) {
            const long long d = (long long)vol[c] - target;
            v2 += d * d;
            v1 += d;
        }
    }
    v2 = warp_sum(v2);
    v1 = warp_sum(v1);
    if ((threadIdx.x & 31) == 0) {
        r2[threadIdx.x >> 5] = v2;
        r1[threadIdx.x >> 5] = v1;
    }
    __syncthreads();
    const int npair = nt * (nt + 1) / 2;
    for (int k = threadIdx.x; k < npair; k += blockDim.x) atomic_add_i64(out + k, scnt[k]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long a2 = 0, a1 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a2 += r2[w];
            a1 += r1[w];
        }
        out[npair] = a2;
        out[npair + 1] = a1;
    }
}

__global__ void __launch_bounds__(1024) finalize_kernel(DevState *state, StatsBufs st, int record) {
    long long slot = (record && st.cap > 0) ? state->n_rec % st.cap : -1;
    if (!SPIN_CK(slot < (long long)st.cap && state->n_rec >= 0, 141)) slot = -1;
    const int n = st.n_lat * st.width;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int64_t v = st.cur[k] + st.delta[k];
        st.cur[k] = v;
        st.delta[k] = 0;
        if (slot >= 0) st.ring[slot * n + k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        state->t += 1;
        if (record) state->n_rec += 1;
    }
}

// Exact moments over records: one block per lattice, threads split the
// records; out is __int128 [n_lat][n_mom] with n_mom = 1 + w + w(w+1)/2.
__global__ void __launch_bounds__(256) moments_kernel(const int64_t *ring, int cap, int n_lat,
                                                      int width, long long first, int n,
                                                      __int128 *out) {
    __shared__ __int128 part[8];
    const int lat = blockIdx.x;
    const int n_mom = 1 + width + width * (width + 1) / 2;
    for (int k = 0; k < n_mom; ++k) {
        int ia = -1, ib = -1;
        if (k >= 1 && k <= width) {
            ia = k - 1;
        } else if (k > width) {
            int r = k - 1 - width, a = 0;
            while (r >= width - a) {
                r -= width - a;
                ++a;
            }
            ia = a;
            ib = a + r;
        }
        __int128 acc = 0;
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const long long rec = first + s;
            const int64_t *row = ring + ((rec % cap) * n_lat + lat) * (long long)width;
            if (k == 0)
                acc += 1;
            else if (ib < 0)
                acc += (__int128)row[ia];
            else
                acc += (__int128)row[ia] * (__int128)row[ib];
        }
        // warp reduction of a 128-bit value as two 64-bit halves with carry
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long lo = (unsigned long long)acc;
            const long long hi = (long long)(acc >> 64);
            const unsigned long long olo = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
            const long long ohi = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
            acc += (((__int128)ohi) << 64) | (__int128)olo;
        }
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            __int128 t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
            out[(size_t)lat * n_mom + k] = t;
        }
        __syncthreads();
    }
}

// Sum of moment rows over lattices (pooled samples of chains sharing theta).
__global__ void pool_moments_kernel(const __int128 *in, int n_lat, int n_mom, __int128 *out) {
    for (int k = threadIdx.x; k < n_mom; k += blockDim.x) {
        __int128 t = 0;
        for (int l = 0; l < n_lat; ++l) t += in[(size_t)l * n_mom + k];
        out[k] = t;
    }
}

// Pooled int128 moments <-> four 32-bit limbs held in int64 words,
// v = l0 + l1 2^32 + l2 2^64 + l3 2^96 with l0..l2 in [0, 2^32) and l3
// signed, so that an element-wise integer sum over ranks stays exact; the
// recombination accepts any int64 limbs (the carries of such a sum).
__global__ void i128_to_limbs_kernel(const __int128 *in, int n, int64_t *limbs) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const __int128 v = in[k];
        const unsigned __int128 u = (unsigned __int128)v;
        limbs[4 * k] = (int64_t)(uint32_t)(u & 0xFFFFFFFFu);
        limbs[4 * k + 1] = (int64_t)(uint32_t)((u >> 32) & 0xFFFFFFFFu);
        limbs[4 * k + 2] = (int64_t)(uint32_t)((u >> 64) & 0xFFFFFFFFu);
        limbs[4 * k + 3] = (int64_t)(v >> 96);
    }
}

__global__ void limbs_to_i128_kernel(const int64_t *limbs, int n, __int128 *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        __int128 v = (__int128)limbs[4 * k + 3];
        v = v * ((__int128)1 << 32) + (__int128)limbs[4 * k + 2];
        v = v * ((__int128)1 << 32) + (__int128)limbs[4 * k + 1];
        v = v * ((__int128)1 << 32) + (__int128)limbs[4 * k];
        out[k] = v;
    }
}

__device__ __forceinline__ double i128_to_double(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double d = (double)(unsigned long long)(u >> 64) * 18446744073709551616.0 +
                     (double)(unsigned long long)(u & 0xFFFFFFFFFFFFFFFFull);
    return neg ? -d : d;
}

__global__ void observables_kernel(const int64_t *ring, int cap, long long first, int n,
                                   ObsParams p, int64_t *stats_out, float *E, float *M) {
    const int total = n * p.n_lat;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int s = idx / p.n_lat, lat = idx - s * p.n_lat;
        const long long rec = first + s;
        const int64_t *row = ring + ((rec % cap) * p.n_lat + lat) * (long long)p.width;
        if (stats_out)
            for (int k = 0; k < p.width; ++k) stats_out[(size_t)idx * p.width + k] = row[k];
        const double *lp = p.lat_params + kLatParams * lat;
        const double J = lp[0], h = lp[1], N = lp[2];
        double e, m;
        if (p.model == 0) {
            const double b2 = p.width > 2 ? lp[4] * (double)row[2] : 0.0;
            e = (-J * (double)row[1] - b2 - h * (double)row[0]) / N;
            m = (double)row[0] / N;
        } else if (p.model == 1) {
            const int q = (int)lp[3];
            long long mx = 0;
            for (int k = 0; k < q; ++k) mx = row[1 + k] > mx ? row[1 + k] : mx;
            e = -J * (double)row[0] / N;
            m = ((double)q * (double)mx - N) / ((double)(q - 1) * N);
        } else {
            const int npair = p.width - 2;
            double adh = 0.0;
            for (int k = 0; k < npair; ++k) adh += p.cpm_J[k] * (double)row[k];
            e = (adh + p.cpm_lambda * (double)row[npair]) / N;
            m = adh / N;
        }
        if (E) E[idx] = (float)e;
        if (M) M[idx] = (float)m;
    }
}

// Covariance of X_i, X_j from exact moments: (n S_ij - S_i S_j) / n^2.
__device__ double cov_ij(const __int128 *mo, int width, int i, int j) {
    if (i > j) {
        const int t = i;
        i = j;
        j = t;
    }
    const __int128 n = mo[0];
    const __int128 Si = mo[1 + i], Sj = mo[1 + j];
    // index of (i, j) in the upper triangle
    const int tri = i * width - i * (i - 1) / 2 + (j - i);
    const __int128 Sij = mo[1 + width + tri];
    const __int128 num = n * Sij - Si * Sj;
    const double nd = (double)(long long)n;
    return i128_to_double(num) / (nd * nd);
}

// One thread per output row; rows are lattices (or one pooled row), lat0 gives
// the parameters of each row.
__global__ void grad_kernel(const __int128 *moments, int rows, GradParams p, double *out) {
    const int width = p.width;
    const int n_mom = 1 + width + width * (width + 1) / 2;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const __int128 *mo = moments + (size_t)row * n_mom;
    const int lat0 = p.pool ? 0 : row;
    const double nd = (double)(long long)mo[0];
    if (p.model == 0) {
        // X = (M, B[, B2]); theta = (J, h[, J2]) with dH/dtheta = -X_{(1, 0, 2)}.
        // O = E/N = (-J B - h M - J2 B2)/N (explicit dO/dtheta = -X_theta / N) or M/N.
        const double *lp = p.lat_params + kLatParams * lat0;
        const double J = lp[0], h = lp[1], N = lp[2], beta = lp[3], J2 = lp[4];
        const int xi[3] = {1, 0, 2};
        for (int j = 0; j < width; ++j) {
            const int k = xi[j];
            double cOX;   // Cov(O, X_k)
            if (p.observable == 0) {
                cOX = -J * cov_ij(mo, width, 1, k) - h * cov_ij(mo, width, 0, k);
                if (width > 2) cOX -= J2 * cov_ij(mo, width, 2, k);
                cOX /= N;
            } else {
                cOX = cov_ij(mo, width, 0, k) / N;
            }
            const double explicit_term = p.observable == 0 ? -i128_to_double(mo[1 + k]) / nd / N : 0.0;
            out[(size_t)width * row + j] = explicit_term - beta * (-cOX);
        }
    } else {
        const int npair = p.n_pairs;
        const double N = p.lat_params[2], beta = 1.0 / p.cpm_T;
        // Cov(O, X_k) with O = sum_a J_a C_a / N
        for (int k = 0; k < npair + 2; ++k) {
            double c = 0.0;
            for (int a = 0; a < npair; ++a) c += p.cpm_J[a] * cov_ij(mo, width, a, k);
            c /= N;
            double g;
            if (k < npair)
                g = i128_to_double(mo[1 + k]) / nd / N - beta * c;   // d/dJ_ab
            else if (k == npair)
                g = -beta * c;                                        // d/dlambda
            else
                g = -beta * (-2.0 * p.cpm_lambda * c);                // d/dA
            out[(size_t)row * (npair + 2) + k] = g;
        }
    }
}

// <E>/N and <M>/N from exact moments (Ising: X = (M, B); CPM: X = (C.., V2, V1)).
__global__ void expectations_kernel(const __int128 *moments, int rows, GradParams p, double *out) {
    const int width = p.width;
    const int n_mom = 1 + width + width * (width + 1) / 2;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const __int128 *mo = moments + (size_t)row * n_mom;
    const int lat0 = p.pool ? 0 : row;
    const double nd = (double)(long long)mo[0];
    if (p.model == 0) {
        const double *lp = p.lat_params + kLatParams * lat0;
        const double J = lp[0], h = lp[1], N = lp[2];
        const double mM = i128_to_double(mo[1]) / nd, mB = i128_to_double(mo[2]) / nd;
        const double mB2 = width > 2 ? i128_to_double(mo[3]) / nd : 0.0;
        out[2 * row] = (-J * mB - lp[4] * mB2 - h * mM) / N;
        out[2 * row + 1] = mM / N;
    } else {
        const int npair = p.n_pairs;
        const double N = p.lat_params[2];
        double adh = 0.0;
        for (int a = 0; a < npair; ++a) adh += p.cpm_J[a] * i128_to_double(mo[1 + a]);
        adh /= nd;
        out[2 * row] = (adh + p.cpm_lambda * i128_to_double(mo[1 + npair]) / nd) / N;
        out[2 * row + 1] = adh / N;
    }
}

__global__ void i128_to_i64_kernel(const __int128 *in, int64_t *out, int n, int *overflow) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const __int128 v = in[i];
        if (v > (__int128)0x7FFFFFFFFFFFFFFFll || v < -(__int128)0x7FFFFFFFFFFFFFFFll) atomicExch(overflow, 1);
        out[i] = (int64_t)v;
    }
}

}  // namespace

cudaError_t launch_stats_from_state(const void *spins, int model, const LatDev *lats, int n_lat,
                                    int maxL, int width, const uint8_t *cpm_type, int cpm_ntypes,
                                    const int32_t *cpm_vol, int cpm_ncells, int cpm_target,
                                    int64_t *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t) * (size_t)n_lat * width, s);
    if (e) return e;
    if (model == 2) {
        const int blocks = (maxL * maxL + 255) / 256;
        stats_cpm_kernel<<<blocks < 512 ? blocks : 512, 256, 0, s>>>(
            static_cast<const int32_t *>(spins), maxL, cpm_type, cpm_ntypes, cpm_vol, cpm_ncells,
            cpm_target, width, out);
    } else {
        const int blocks = (maxL * maxL + 255) / 256;
        dim3 grid(blocks < 128 ? blocks : 128, n_lat);
        stats_state_kernel<<<grid, 256, 0, s>>>(spins, model, lats, width, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(DevState *state, StatsBufs st, int record, cudaStream_t s) {
    finalize_kernel<<<1, 1024, 0, s>>>(state, st, record);
    return cudaGetLastError();
}

cudaError_t launch_moments_i128(const StatsBufs &st, int64_t first, int n, void *out,
                                cudaStream_t s) {
    moments_kernel<<<st.n_lat, 256, 0, s>>>(st.ring, st.cap, st.n_lat, st.width, first, n,
                                            static_cast<__int128 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_pool_moments(const void *in, int n_lat, int n_mom, void *out, cudaStream_t s) {
    pool_moments_kernel<<<1, 256, 0, s>>>(static_cast<const __int128 *>(in), n_lat, n_mom,
                                          static_cast<__int128 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_i128_to_limbs(const void *in, int n, int64_t *limbs, cudaStream_t s) {
    i128_to_limbs_kernel<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const __int128 *>(in), n, limbs);
    return cudaGetLastError();
}

cudaError_t launch_limbs_to_i128(const int64_t *limbs, int n, void *out, cudaStream_t s) {
    limbs_to_i128_kernel<<<(n + 255) / 256, 256, 0, s>>>(limbs, n, static_cast<__int128 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_i128_to_i64(const void *in, int64_t *out, int n, int *overflow, cudaStream_t s) {
    i128_to_i64_kernel<<<(n + 255) / 256, 256, 0, s>>>(static_cast<const __int128 *>(in), out, n,
                                                       overflow);
    return cudaGetLastError();
}

cudaError_t launch_observables(const StatsBufs &st, int64_t first, int n, ObsParams p,
                               int64_t *stats_out, float *E, float *M, cudaStream_t s) {
    const int total = n * p.n_lat;
    int blocks = (total + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks);
    observables_kernel<<<blocks, 256, 0, s>>>(st.ring, st.cap, first, n, p, stats_out, E, M);
    return cudaGetLastError();
}

cudaError_t launch_expectations_i128(const void *moments, int rows, GradParams p, double *out,
                                     cudaStream_t s) {
    expectations_kernel<<<(rows + 63) / 64, 64, 0, s>>>(static_cast<const __int128 *>(moments), rows, p,
                                                        out);
    return cudaGetLastError();
}

cudaError_t launch_grad_i128(const void *moments, int rows, GradParams p, double *out,
                             cudaStream_t s) {
    grad_kernel<<<(rows + 63) / 64, 64, 0, s>>>(static_cast<const __int128 *>(moments), rows, p, out);
    return cudaGetLastError();
}

// ------------------------------------------------------ bit-packed host transfer
namespace {

// Four sign bits (bit 7 of each byte) gathered into a nibble: the products of
// the masked bits with 1 + 2^7 + 2^14 + 2^21 land on distinct positions, so
// bits 28..31 are the four signs in byte order.
__device__ __forceinline__ uint32_t sign_nibble(uint32_t w) { return ((w & 0x80808080u) * 0x00204081u) >> 28; }

// The inverse: four bits -> four bytes 0x01 (bit 0) / 0xFF (bit 1).
__device__ __forceinline__ uint32_t nibble_bytes(uint32_t n) {
    const uint32_t spread = (n * 0x00204081u) & 0x01010101u;
    return 0x01010101u + spread * 0xFEu;
}

// Sides the row-strip kernel takes (with skip_strip, the pack and unpack
// kernels leave those lattices' spins to the strip kernel's bit layouts).
__device__ __forceinline__ bool strip_side(int L) { return L == 512 || L == 1024 || L == 2048; }

// The blocks of a pack or unpack launch are cut per lattice: lattice l owns
// blocks [blk[l], blk[l + 1]) (a host-built prefix of per-lattice counts that
// follow its word count, so small lattices take one block and no block idles).
// Block b finds its lattice by bisection.
__device__ __forceinline__ int block_lattice(const int32_t *blk, int n_lat, int b) {
    int lo = 0, hi = n_lat - 1;   // the last lattice whose first block is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One thread per 32-bit word of the packed buffer overlapping its lattice
// (offsets are multiples of 32, so no word holds two lattices).
__global__ void pack_spins_kernel(const int8_t *spins, uint32_t *words, const LatDev *lats, const int32_t *blk,
                                  int n_lat, int skip_strip) {
    const int lat = block_lattice(blk, n_lat, (int)blockIdx.x);
    const int lb = (int)blockIdx.x - blk[lat], nb = blk[lat + 1] - blk[lat];
    const LatDev ld = lats[lat];
    if (skip_strip && strip_side(ld.L)) return;
    const size_t o = ld.offset, end = o + (size_t)ld.L * ld.L;
    for (size_t w = (o >> 5) + lb * (size_t)blockDim.x + threadIdx.x; (w << 5) < end;
         w += (size_t)nb * blockDim.x) {
        const size_t e0 = w << 5;
        uint32_t bits = 0;
        if (e0 + 32 <= end && ((reinterpret_cast<uintptr_t>(spins + e0) & 15) == 0)) {
            const uint4 a = *reinterpret_cast<const uint4 *>(spins + e0);
            const uint4 b = *reinterpret_cast<const uint4 *>(spins + e0 + 16);
            const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) bits |= sign_nibble(v[k]) << (4 * k);
        } else {
            for (int i = 0; i < 32 && e0 + i < end; ++i)
                if (spins[e0 + i] < 0) bits |= 1u << i;
        }
        words[w] = bits;
    }
}

// Bit of element e (1: the spin is -1).
__device__ __forceinline__ int packed_bit(const uint32_t *words, size_t e) { return (words[e >> 5] >> (e & 31)) & 1; }

// Unpack, and count the statistics of the loaded state on the way (cur must be
// zero on entry): M = sum s, B = sum over right and down bonds of s s'.  Rows
// of 32k spins are whole words: a word's right neighbours are its bits shifted
// by one with bit 0 of the next word of the row (or of the row's first word),
// its down neighbours the word of the next row, and unequal pairs are popcounts
// of xors.  Other sides count bond by bond.
__global__ void unpack_spins_kernel(const uint32_t *words, int8_t *spins, const LatDev *lats, const int32_t *blk,
                                    int n_lat, int64_t *cur, int skip_strip) {
    __shared__ long long red[2][8];
    const int lat = block_lattice(blk, n_lat, (int)blockIdx.x);
    const int lb = (int)blockIdx.x - blk[lat], nb = blk[lat + 1] - blk[lat];
    const LatDev ld = lats[lat];
    const int L = ld.L;
    const bool write = !(skip_strip && strip_side(L));   // else statistics only
    const size_t o = ld.offset, end = o + (size_t)L * L;
    const bool rows_whole = (L & 31) == 0;
    const int wpr = L >> 5;   // words per row when rows_whole
    // spin_offset % 32 == 0: word wl of the lattice is global word (o >> 5) + wl.
    // (r, q) = (row, word in the row) of wl, advanced by the grid stride as rows
    // and words instead of dividing
    const uint32_t n_wl = (uint32_t)(((size_t)L * L + 31) >> 5);
    const uint32_t stride = (uint32_t)nb * blockDim.x;
    uint32_t wl = (uint32_t)lb * blockDim.x + threadIdx.x;
    int r = 0, q = 0, dr = 0, dq = 0;
    if (rows_whole) {
        r = (int)(wl / (uint32_t)wpr);
        q = (int)wl - r * wpr;
        dr = (int)(stride / (uint32_t)wpr);
        dq = (int)stride - dr * wpr;
    }
    int m = 0, b = 0;   // at most 32 (m) and 64 (b) per word, a few thousand words per thread
    for (; wl < n_wl; wl += stride) {
        const size_t w = (o >> 5) + wl;
        const size_t e0 = w << 5;
        const uint32_t bits = words[w];
        if (!write) {
        } else if (e0 + 32 <= end && ((reinterpret_cast<uintptr_t>(spins + e0) & 15) == 0)) {
            uint32_t v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = nibble_bytes((bits >> (4 * k)) & 0xFu);
            *reinterpret_cast<uint4 *>(spins + e0) = make_uint4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<uint4 *>(spins + e0 + 16) = make_uint4(v[4], v[5], v[6], v[7]);
        } else {
            for (int i = 0; i < 32 && e0 + i < end; ++i) spins[e0 + i] = ((bits >> i) & 1u) ? -1 : 1;
        }
        if (!cur) continue;
        if (rows_whole) {
            const size_t row0 = (o >> 5) + (size_t)r * wpr;
            const uint32_t nxt = words[row0 + (q + 1 == wpr ? 0 : q + 1)];
            const uint32_t right = (bits >> 1) | (nxt << 31);
            const uint32_t down = words[(o >> 5) + (size_t)(r + 1 == L ? 0 : r + 1) * wpr + q];
            m += 32 - 2 * __popc(bits);
            b += 64 - 2 * (__popc(bits ^ right) + __popc(bits ^ down));
            r += dr;
            q += dq;
            if (q >= wpr) {
                q -= wpr;
                ++r;
            }
        } else {
            for (int i = 0; i < 32 && e0 + i < end; ++i) {
                const size_t e = e0 + i, k = e - o;
                const int y = (int)(k / L), x = (int)(k - (size_t)y * L);
                const int sb = packed_bit(words, e);
                const int rb = packed_bit(words, o + (size_t)y * L + (x + 1 == L ? 0 : x + 1));
                const int db = packed_bit(words, o + (size_t)(y + 1 == L ? 0 : y + 1) * L + x);
                m += 1 - 2 * sb;
                b += (sb == rb ? 1 : -1) + (sb == db ? 1 : -1);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m += __shfl_xor_sync(0xFFFFFFFFu, m, off);
        b += __shfl_xor_sync(0xFFFFFFFFu, b, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = m;
        red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0 && cur) {
        long long tm = 0, tb = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            tm += red[0][k];
            tb += red[1][k];
        }
        if (tm) atomicAdd(reinterpret_cast<unsigned long long *>(cur + 2 * lat), (unsigned long long)tm);
        if (tb) atomicAdd(reinterpret_cast<unsigned long long *>(cur + 2 * lat + 1), (unsigned long long)tb);
    }
}

}  // namespace

cudaError_t launch_unpack_spins(const uint32_t *words, int8_t *spins, const LatDev *lats, int n_lat,
                                const int32_t *blk, int n_blocks, int64_t *cur, cudaStream_t s, bool skip_strip) {
    if (cur) {
        cudaError_t e = cudaMemsetAsync(cur, 0, sizeof(int64_t) * 2 * (size_t)n_lat, s);
        if (e) return e;
    }
    if (n_blocks <= 0) return cudaSuccess;
    unpack_spins_kernel<<<n_blocks, 256, 0, s>>>(words, spins, lats, blk, n_lat, cur, skip_strip ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_pack_spins(const int8_t *spins, uint32_t *words, size_t n_words, const LatDev *lats, int n_lat,
                              const int32_t *blk, int n_blocks, cudaStream_t s, bool skip_strip) {
    if (!skip_strip) {   // with skip_strip the caller keeps the other words (cleared, or written by the strip kernel)
        cudaError_t e = cudaMemsetAsync(words, 0, n_words * sizeof(uint32_t), s);
        if (e) return e;
    }
    if (n_blocks <= 0) return cudaSuccess;
    pack_spins_kernel<<<n_blocks, 256, 0, s>>>(spins, words, lats, blk, n_lat, skip_strip ? 1 : 0);
    return cudaGetLastError();
}

SPIN_CHECK_ACCESSOR(check_word_stats)

}  // namespace spinmc
