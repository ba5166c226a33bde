/*
 * spin_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the checkerboard
 * Metropolis-Hastings method of "A differentiable programming framework for
 * spin models" (Farias, Schultz, Mombach, Maziero; arXiv 2304.01772).  Only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, table or helper with the CUDA library:
 * every rule below is written out again from the paper and from the fixed
 * conventions that the paper leaves open (listed in each function's comment).
 *
 * Everything is computed site by site, in the order the paper describes:
 * colour sub-steps of the checkerboard (Sec. "Related Work", checkerboard
 * figure; Alg. 1), a proposal, the local energy change, and the Metropolis
 * acceptance (Alg. 1: accept when dE <= 0, else with p = exp(-beta*dE)).
 *
 * Conventions fixed where the paper is silent or ambiguous (the paper prints
 * H = sum J s_i s_j + sum B s_i with J < 0 ferromagnetic, Eq. of Sec. "Ising
 * model"; this code uses the equivalent standard form):
 *   Ising  H = -J sum_<ij> s_i s_j - h sum_i s_i, each bond once, s = +-1.
 *   Potts  H = -J sum_<ij> delta(s_i, s_j), s in {0..q-1}, no field.
 *   CPM    H = sum_<xy> J(tau(s_x), tau(s_y)) (1 - delta(s_x, s_y))
 *              + lambda sum_{cells != 0} (a_s - A)^2      (Eq. "h"),
 *          unordered Moore pairs (8 neighbours) counted once.
 *   Random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *     key = (seed_lo, seed_hi), counter = (g, lattice, sweep, colour).
 *   Acceptance of a draw u (uint32): dE <= 0 always; otherwise
 *     u < max(floor(exp(-beta*dE) * 2^32), 1).
 *
 * parity pinned: Philox by published known-answer vectors; the chains by
 * exact enumeration (4x4), Onsager's solution, detailed balance, the q=2
 * Potts/Ising identity and CPM bookkeeping invariants; the differentiable
 * Monte Carlo of Alg. 2 by finite differences of its forward pass, its
 * alpha -> infinity Metropolis limit and a closed form; the triangular and
 * the first-and-second-neighbour lattices by brute-force replicas over
 * independently built bond lists and exact enumeration (see tests/).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10, Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of the   */
/* counter words 0 and 2 with fixed multipliers; the high halves are    */
/* xor-ed with the other counter words and the round key; the key is    */
/* bumped by the Weyl constants between rounds.                          */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block for (seed; g, lattice, sweep, colour). */
static void draw4(uint64_t seed, uint32_t g, uint32_t lattice, uint32_t sweep,
                  uint32_t colour, uint32_t out[4])
{
    uint32_t ctr[4] = {g, lattice, sweep, colour};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* XOR of all four words of the blocks for counters (g, lattice, sweep,
 * colour), g = g0 .. g0 + n - 1: a digest of one stretch of the random
 * stream that the sweeps draw from. */
uint32_t or_philox_xor(uint64_t seed, uint32_t lattice, uint32_t sweep, uint32_t colour,
                       uint32_t g0, uint32_t n)
{
    uint32_t acc = 0, out[4];
    for (uint32_t i = 0; i < n; ++i) {
        draw4(seed, g0 + i, lattice, sweep, colour, out);
        acc ^= out[0] ^ out[1] ^ out[2] ^ out[3];
    }
    return acc;
}

/* floor(u * m / 2^32): an index in [0, m) from a uniform uint32. */
static uint32_t mulhi32(uint32_t u, uint32_t m)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)m) >> 32);
}

/* ------------------------------------------------------------------ */
/* Metropolis acceptance (Alg. 1): accept if dE <= 0, else with         */
/* probability exp(-beta dE), quantised to k/2^32 with k >= 1.          */
/* ------------------------------------------------------------------ */
double or_accept_count(double beta, double dE)
{
    /* Number of the 2^32 values of u that are accepted. */
    if (dE <= 0.0) return 4294967296.0;
    double p = exp(-beta * dE);
    double k = floor(p * 4294967296.0);
    if (k < 1.0) k = 1.0;
    if (k > 4294967296.0) k = 4294967296.0;
    return k;
}

int or_accept(double beta, double dE, uint32_t u)
{
    return (double)u < or_accept_count(beta, dE);
}

static int wrap(int i, int L) { return ((i % L) + L) % L; }

/* ------------------------------------------------------------------ */
/* Initial states.  Random initial lattice (Sec. "Related Work": a      */
/* random initial state is chosen).  Draw for site i = y*L + x:          */
/* Philox(seed; g = i >> 2, lattice, 0xFFFFFFFF, 0), lane i & 3.         */
/* ------------------------------------------------------------------ */
static uint32_t init_draw(uint64_t seed, uint32_t lattice, uint32_t i)
{
    uint32_t r[4];
    draw4(seed, i >> 2, lattice, 0xFFFFFFFFu, 0u, r);
    return r[i & 3u];
}

void or_init_ising(int L, uint64_t seed, uint32_t lattice, int8_t *s)
{
    for (int i = 0; i < L * L; ++i) {
        uint32_t u = init_draw(seed, lattice, (uint32_t)i);
        s[i] = (u >> 31) ? (int8_t)1 : (int8_t)-1;
    }
}

void or_init_potts(int L, int q, uint64_t seed, uint32_t lattice, uint8_t *s)
{
    for (int i = 0; i < L * L; ++i) {
        uint32_t u = init_draw(seed, lattice, (uint32_t)i);
        s[i] = (uint8_t)mulhi32(u, (uint32_t)q);
    }
}

/* ------------------------------------------------------------------ */
/* Ising colour sub-step and sweep (Alg. 1 with the 4-neighbour stencil */
/* K of Sec. "Ising model").  Colour of (x, y) is (x + y) & 1; colour 0  */
/* is updated first.  The proposal is the flip s -> -s.  The draw of     */
/* site (x, y) of colour c: k = (y*L + x) >> 1, Philox(seed; k >> 2,     */
/* lattice, sweep, c), lane k & 3.                                       */
/* ------------------------------------------------------------------ */
void or_ising_substep(int L, float beta, float J, float h, uint64_t seed,
                      uint32_t lattice, uint32_t sweep, int colour, int8_t *s)
{
    double beta_d = (double)beta;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            if (((x + y) & 1) != colour) continue;
            int sig = s[y * L + x];
            int n = s[wrap(y - 1, L) * L + x] + s[wrap(y + 1, L) * L + x]
                  + s[y * L + wrap(x - 1, L)] + s[y * L + wrap(x + 1, L)];
            /* H = -J sum s s - h sum s: flipping s changes H by 2 s (J n + h). */
            double dE = 2.0 * (double)sig * ((double)J * (double)n + (double)h);
            uint32_t k = (uint32_t)(y * L + x) >> 1;
            uint32_t r[4];
            draw4(seed, k >> 2, lattice, sweep, (uint32_t)colour, r);
            if (or_accept(beta_d, dE, r[k & 3u])) s[y * L + x] = (int8_t)(-sig);
        }
    }
}

void or_ising_sweep(int L, float beta, float J, float h, uint64_t seed,
                    uint32_t lattice, uint32_t sweep, int8_t *s)
{
    or_ising_substep(L, beta, J, h, seed, lattice, sweep, 0, s);
    or_ising_substep(L, beta, J, h, seed, lattice, sweep, 1, s);
}

/* M = sum s, B = sum over bonds (right and down of every site) s s'. */
void or_ising_stats(int L, const int8_t *s, int64_t out[2])
{
    int64_t M = 0, B = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int v = s[y * L + x];
            M += v;
            B += v * s[y * L + wrap(x + 1, L)];
            B += v * s[wrap(y + 1, L) * L + x];
        }
    out[0] = M;
    out[1] = B;
}

/* n sweeps starting at sweep index sweep0; stats after each sweep. */
void or_ising_run(int L, float beta, float J, float h, uint64_t seed, uint32_t lattice,
                  uint32_t sweep0, int nsweeps, int8_t *s, int64_t *stats)
{
    for (int t = 0; t < nsweeps; ++t) {
        or_ising_sweep(L, beta, J, h, seed, lattice, sweep0 + (uint32_t)t, s);
        if (stats) or_ising_stats(L, s, stats + 2 * (size_t)t);
    }
}

/* ------------------------------------------------------------------ */
/* Potts colour sub-step (Eq. of Sec. "Potts model"; proposal: one of    */
/* the q-1 other values, s' = (s + 1 + floor(u1 (q-1) / 2^32)) mod q).   */
/* Site draw: k = (y*L + x) >> 1, Philox(seed; k >> 1, lattice, sweep,   */
/* c), lanes 2(k&1) (acceptance u0) and 2(k&1)+1 (choice u1).            */
/* dE = J (n_same(s) - n_same(s')) for H = -J sum delta.                 */
/* ------------------------------------------------------------------ */
void or_potts_substep(int L, int q, float beta, float J, uint64_t seed,
                      uint32_t lattice, uint32_t sweep, int colour, uint8_t *s)
{
    double beta_d = (double)beta;
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            if (((x + y) & 1) != colour) continue;
            int sig = s[y * L + x];
            int nb[4] = {s[wrap(y - 1, L) * L + x], s[wrap(y + 1, L) * L + x],
                         s[y * L + wrap(x - 1, L)], s[y * L + wrap(x + 1, L)]};
            uint32_t k = (uint32_t)(y * L + x) >> 1;
            uint32_t r[4];
            draw4(seed, k >> 1, lattice, sweep, (uint32_t)colour, r);
            uint32_t u0 = r[2u * (k & 1u)], u1 = r[2u * (k & 1u) + 1u];
            int sp = (int)(((uint32_t)sig + 1u + mulhi32(u1, (uint32_t)(q - 1))) % (uint32_t)q);
            int n_old = 0, n_new = 0;
            for (int j = 0; j < 4; ++j) {
                n_old += (nb[j] == sig);
                n_new += (nb[j] == sp);
            }
            double dE = (double)J * (double)(n_old - n_new);
            if (or_accept(beta_d, dE, u0)) s[y * L + x] = (uint8_t)sp;
        }
    }
}

void or_potts_sweep(int L, int q, float beta, float J, uint64_t seed,
                    uint32_t lattice, uint32_t sweep, uint8_t *s)
{
    or_potts_substep(L, q, beta, J, seed, lattice, sweep, 0, s);
    or_potts_substep(L, q, beta, J, seed, lattice, sweep, 1, s);
}

/* out[0] = number of equal nearest-neighbour bonds; out[1 + k] = n_k. */
void or_potts_stats(int L, int q, const uint8_t *s, int64_t *out)
{
    for (int k = 0; k <= q; ++k) out[k] = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int v = s[y * L + x];
            out[0] += (v == s[y * L + wrap(x + 1, L)]);
            out[0] += (v == s[wrap(y + 1, L) * L + x]);
            out[1 + v] += 1;
        }
}

void or_potts_run(int L, int q, float beta, float J, uint64_t seed, uint32_t lattice,
                  uint32_t sweep0, int nsweeps, uint8_t *s, int64_t *stats)
{
    for (int t = 0; t < nsweeps; ++t) {
        or_potts_sweep(L, q, beta, J, seed, lattice, sweep0 + (uint32_t)t, s);
        if (stats) or_potts_stats(L, q, s, stats + (size_t)(q + 1) * (size_t)t);
    }
}

/* ------------------------------------------------------------------ */
/* Cellular Potts model (Sec. "Cellular Potts model", Eq. "h").          */
/* Copy attempt: target x, a random Moore neighbour y, proposal          */
/* s(x) <- s(y), decided by Alg. 1.  Sites are coloured                  */
/* c = (x & 1) | ((y & 1) << 1) so that no two sites of one colour are   */
/* Moore neighbours; colours 0..3 in order make one Monte Carlo step.    */
/* Site draw: k = (y >> 1)*(L/2) + (x >> 1), Philox(seed; k >> 1,         */
/* lattice, sweep, c), lanes 2(k&1) (u0, acceptance) and 2(k&1)+1 (u1,    */
/* neighbour choice u1 >> 29 in the order below).  Area terms use the    */
/* cell areas as they stood at the start of the colour sub-step;         */
/* accepted copies change the areas for the next sub-step.  Medium (id 0) */
/* has no area term.                                                     */
/* ------------------------------------------------------------------ */
static const int moore_dx[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int moore_dy[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

typedef struct {
    int n_types;
    const int32_t *J;          /* n_types x n_types, symmetric */
    int lambda;
    int target;
    int n_cells;               /* ids 1..n_cells, 0 = medium */
    const uint8_t *type;       /* [n_cells + 1], type[0] = 0 */
    float T;
} or_cpm;

static int cpm_J(const or_cpm *p, int a, int b) { return p->J[a * p->n_types + b]; }

/* Area energy of a cell with area a (0 for the medium). */
static int64_t area_energy(const or_cpm *p, int id, int64_t a)
{
    if (id == 0) return 0;
    int64_t d = a - p->target;
    return (int64_t)p->lambda * d * d;
}

void or_cpm_substep(int L, int n_types, const int32_t *Jtab, int lambda, int target,
                    int n_cells, const uint8_t *type, float T, uint64_t seed,
                    uint32_t lattice, uint32_t sweep, int colour, int32_t *id, int32_t *vol)
{
    or_cpm p = {n_types, Jtab, lambda, target, n_cells, type, T};
    int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_cells + 1));
    memcpy(snap, vol, sizeof(int32_t) * (size_t)(n_cells + 1));
    for (int y = 0; y < L; ++y) {
        for (int x = 0; x < L; ++x) {
            if (((x & 1) | ((y & 1) << 1)) != colour) continue;
            uint32_t k = (uint32_t)((y >> 1) * (L / 2) + (x >> 1));
            uint32_t r[4];
            draw4(seed, k >> 1, lattice, sweep, (uint32_t)colour, r);
            uint32_t u0 = r[2u * (k & 1u)], u1 = r[2u * (k & 1u) + 1u];
            int nbi = (int)(u1 >> 29);
            int sg = id[y * L + x];
            int sp = id[wrap(y + moore_dy[nbi], L) * L + wrap(x + moore_dx[nbi], L)];
            if (sp == sg) continue;
            /* Adhesion: only the 8 pairs (x, z) change. */
            int64_t dH = 0;
            for (int j = 0; j < 8; ++j) {
                int sz = id[wrap(y + moore_dy[j], L) * L + wrap(x + moore_dx[j], L)];
                if (sz != sp) dH += cpm_J(&p, type[sp], type[sz]);
                if (sz != sg) dH -= cpm_J(&p, type[sg], type[sz]);
            }
            /* Area: sp gains one site, sg loses one (snapshot areas). */
            dH += area_energy(&p, sp, snap[sp] + 1) - area_energy(&p, sp, snap[sp]);
            dH += area_energy(&p, sg, snap[sg] - 1) - area_energy(&p, sg, snap[sg]);
            /* Alg. 1 with p = exp(-dE / T), T the paper's k_B T; the same
             * 2^-32 quantisation as or_accept_count. */
            int accept;
            double dE = (double)dH;
            if (dE <= 0.0) {
                accept = 1;
            } else {
                double kk = floor(exp(-dE / (double)T) * 4294967296.0);
                if (kk < 1.0) kk = 1.0;
                accept = (double)u0 < kk;
            }
            if (accept) {
                id[y * L + x] = sp;
                vol[sp] += 1;
                vol[sg] -= 1;
            }
        }
    }
    free(snap);
}

void or_cpm_sweep(int L, int n_types, const int32_t *Jtab, int lambda, int target,
                  int n_cells, const uint8_t *type, float T, uint64_t seed,
                  uint32_t lattice, uint32_t sweep, int32_t *id, int32_t *vol)
{
    for (int c = 0; c < 4; ++c)
        or_cpm_substep(L, n_types, Jtab, lambda, target, n_cells, type, T, seed,
                       lattice, sweep, c, id, vol);
}

/* Contact counts C[a][b] (a <= b, row-major upper triangle) over unordered
 * Moore pairs of different cells, then V2 = sum_cells (a - A)^2 and
 * V1 = sum_cells (a - A). */
void or_cpm_stats(int L, int n_types, int target, int n_cells, const uint8_t *type,
                  const int32_t *id, const int32_t *vol, int64_t *out)
{
    int npair = n_types * (n_types + 1) / 2;
    for (int i = 0; i < npair + 2; ++i) out[i] = 0;
    /* right, down-left, down, down-right: each unordered pair once. */
    static const int hx[4] = {1, -1, 0, 1};
    static const int hy[4] = {0, 1, 1, 1};
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int a = id[y * L + x];
            for (int j = 0; j < 4; ++j) {
                int b = id[wrap(y + hy[j], L) * L + wrap(x + hx[j], L)];
                if (a == b) continue;
                int ta = type[a], tb = type[b];
                int lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
                int idx = lo * n_types - lo * (lo - 1) / 2 + (hi - lo);
                out[idx] += 1;
            }
        }
    for (int c = 1; c <= n_cells; ++c) {
        int64_t d = (int64_t)vol[c] - target;
        out[npair] += d * d;
        out[npair + 1] += d;
    }
}

/* Initial CPM state: square cells of side `side` on a block grid of `cols`
 * cells per row, centred, ids row-major from 1; medium elsewhere.  Cell
 * types: Philox(seed; g = id, lattice, 0xFFFFFFFE, 0) lane 0, type
 * 1 + (u >> 31) (two cell types, as in the paper's cell-sorting setup). */
int or_cpm_init(int L, int n_cells, int side, int cols, uint64_t seed, uint32_t lattice,
                int32_t *id, uint8_t *type, int32_t *vol)
{
    int rows = (n_cells + cols - 1) / cols;
    int x0 = (L - cols * side) / 2, y0 = (L - rows * side) / 2;
    if (x0 < 0 || y0 < 0) return -1;
    for (int i = 0; i < L * L; ++i) id[i] = 0;
    for (int c = 0; c < n_cells; ++c) {
        int bx = c % cols, by = c / cols;
        for (int dy = 0; dy < side; ++dy)
            for (int dx = 0; dx < side; ++dx)
                id[(y0 + by * side + dy) * L + (x0 + bx * side + dx)] = c + 1;
    }
    type[0] = 0;
    for (int c = 1; c <= n_cells; ++c) {
        uint32_t r[4];
        draw4(seed, (uint32_t)c, lattice, 0xFFFFFFFEu, 0u, r);
        type[c] = (uint8_t)(1u + (r[0] >> 31));
    }
    for (int c = 0; c <= n_cells; ++c) vol[c] = 0;
    for (int i = 0; i < L * L; ++i) vol[id[i]] += 1;
    return 0;
}

void or_cpm_run(int L, int n_types, const int32_t *Jtab, int lambda, int target,
                int n_cells, const uint8_t *type, float T, uint64_t seed, uint32_t lattice,
                uint32_t sweep0, int nsweeps, int32_t *id, int32_t *vol, int64_t *stats)
{
    int width = n_types * (n_types + 1) / 2 + 2;
    for (int t = 0; t < nsweeps; ++t) {
        or_cpm_sweep(L, n_types, Jtab, lambda, target, n_cells, type, T, seed, lattice,
                     sweep0 + (uint32_t)t, id, vol);
        if (stats) or_cpm_stats(L, n_types, target, n_cells, type, id, vol,
                                stats + (size_t)width * (size_t)t);
    }
}

/* Total CPM energy from scratch (Eq. "h"), for the bookkeeping tests. */
int64_t or_cpm_energy(int L, int n_types, const int32_t *Jtab, int lambda, int target,
                      int n_cells, const uint8_t *type, const int32_t *id)
{
    or_cpm p = {n_types, Jtab, lambda, target, n_cells, type, 1.0f};
    int64_t H = 0;
    static const int hx[4] = {1, -1, 0, 1};
    static const int hy[4] = {0, 1, 1, 1};
    int64_t *area = (int64_t *)calloc((size_t)(n_cells + 1), sizeof(int64_t));
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int a = id[y * L + x];
            area[a] += 1;
            for (int j = 0; j < 4; ++j) {
                int b = id[wrap(y + hy[j], L) * L + wrap(x + hx[j], L)];
                if (a != b) H += cpm_J(&p, type[a], type[b]);
            }
        }
    for (int c = 1; c <= n_cells; ++c) H += area_energy(&p, c, area[c]);
    free(area);
    return H;
}

/* ------------------------------------------------------------------ */
/* Differentiable Monte Carlo (Alg. 2, Sec. "Methods"), Ising model    */
/* with one exchange parameter per bond (the J_ij optimised in Sec.     */
/* "Optimization of the exchange parameters").  Relaxed spins s in      */
/* [-1, 1]; Jr[y*L+x] couples (x,y)-(x+1,y), Jd[y*L+x] couples          */
/* (x,y)-(x,y+1), periodic.  Sub-step of colour c, every site i with    */
/* (x+y)&1 == c at once (checkerboard):                                 */
/*   n   = sum_j J_ij s_j            (weighted neighbour sum)           */
/*   dE  = E(s') - E(s) = 2 s (n + h)  for the proposal s' = -s under   */
/*         H = -sum_<ij> J_ij s_i s_j - h sum_i s_i                     */
/*   p   = exp(-beta dE)             (not clipped: Alg. 2 takes it as is)*/
/*   r   = (u >> 8) 2^-24, u the site's Philox lane (Ising layout)      */
/*   q   = 1 / (1 + exp(-alpha (p - r)))                                */
/*   s  <- q s' + (1 - q) s = s (1 - 2 q).                              */
/* The reverse pass is the chain rule through these steps, written by   */
/* hand: with w = dL/ds_new(i) * ds_new/dn,                              */
/*   ds_new/ds = (1 - 2q) + 4 alpha beta p q (1-q) s (n + h)            */
/*   ds_new/dn = 4 alpha beta p q (1-q) s^2                             */
/*   dL/ds_old(j) += w J_ij, dL/dJ_ij += w s_j   (j a neighbour of i).   */
/* parity pinned by central finite differences of the forward pass, the */
/* alpha -> infinity limit (Metropolis with acceptance r < exp(-b dE)),  */
/* and the J = h = 0 closed form (see tests/).                           */
/* ------------------------------------------------------------------ */
static double dmc_r(uint64_t seed, uint32_t lattice, uint32_t sweep, int colour, int L, int x, int y)
{
    uint32_t k = (uint32_t)(y * L + x) >> 1;
    uint32_t r[4];
    draw4(seed, k >> 2, lattice, sweep, (uint32_t)colour, r);
    return (double)(r[k & 3u] >> 8) * (1.0 / 16777216.0);
}

/* Weighted neighbour sum n_i = sum_j J_ij s_j of site (x, y). */
static double dmc_field(int L, const double *Jr, const double *Jd, const double *s, int x, int y)
{
    int xl = wrap(x - 1, L), xr = wrap(x + 1, L), yu = wrap(y - 1, L), yd = wrap(y + 1, L);
    return Jr[y * L + x] * s[y * L + xr] + Jr[y * L + xl] * s[y * L + xl]
         + Jd[y * L + x] * s[yd * L + x] + Jd[yu * L + x] * s[yu * L + x];
}

void or_dmc_substep(int L, const double *Jr, const double *Jd, double beta, double h, double alpha,
                    uint64_t seed, uint32_t lattice, uint32_t sweep, int colour, double *s)
{
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            if (((x + y) & 1) != colour) continue;
            double si = s[y * L + x];
            double n = dmc_field(L, Jr, Jd, s, x, y);
            double dE = 2.0 * si * (n + h);
            double p = exp(-beta * dE);
            double r = dmc_r(seed, lattice, sweep, colour, L, x, y);
            double q = 1.0 / (1.0 + exp(-alpha * (p - r)));
            s[y * L + x] = q * (-si) + (1.0 - q) * si;
        }
}

/* n_sweeps sweeps (colour 0 then 1) starting at sweep index sweep0; tape */
/* (nullable) receives the full state before each of the 2 n_sweeps       */
/* sub-steps, [2 n_sweeps][L*L].                                           */
void or_dmc_run(int L, const double *Jr, const double *Jd, double beta, double h, double alpha,
                uint64_t seed, uint32_t lattice, uint32_t sweep0, int n_sweeps, double *s, double *tape)
{
    for (int t = 0; t < n_sweeps; ++t)
        for (int c = 0; c < 2; ++c) {
            if (tape) memcpy(tape + (size_t)(2 * t + c) * (size_t)(L * L), s, sizeof(double) * (size_t)(L * L));
            or_dmc_substep(L, Jr, Jd, beta, h, alpha, seed, lattice, sweep0 + (uint32_t)t, c, s);
        }
}

/* Reverse pass through the sub-steps recorded in `tape`.  g: on entry     */
/* dL/ds after the last sub-step, on exit dL/ds before the first; gJr, gJd */
/* receive dL/dJ (overwritten).                                            */
void or_dmc_backward(int L, const double *Jr, const double *Jd, double beta, double h, double alpha,
                     uint64_t seed, uint32_t lattice, uint32_t sweep0, int n_sweeps,
                     const double *tape, double *g, double *gJr, double *gJd)
{
    size_t N = (size_t)(L * L);
    double *w = (double *)calloc(N, sizeof(double));
    memset(gJr, 0, sizeof(double) * N);
    memset(gJd, 0, sizeof(double) * N);
    for (int k = 2 * n_sweeps - 1; k >= 0; --k) {
        const double *s = tape + (size_t)k * N;            /* state before sub-step k */
        int colour = k & 1;
        uint32_t sweep = sweep0 + (uint32_t)(k >> 1);
        /* active sites: w_i and the direct term */
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x;
                if (((x + y) & 1) != colour) { w[i] = 0.0; continue; }
                double si = s[i];
                double n = dmc_field(L, Jr, Jd, s, x, y);
                double p = exp(-beta * 2.0 * si * (n + h));
                double r = dmc_r(seed, lattice, sweep, colour, L, x, y);
                double q = 1.0 / (1.0 + exp(-alpha * (p - r)));
                double common = 4.0 * alpha * beta * p * q * (1.0 - q);
                w[i] = g[i] * common * si * si;
                g[i] = g[i] * ((1.0 - 2.0 * q) + common * si * (n + h));
            }
        /* bonds: one end is active (weight w), the other passive */
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = y * L + x;
                int ir = y * L + wrap(x + 1, L), id = wrap(y + 1, L) * L + x;
                /* bond (i, ir) with coupling Jr[i]; bond (i, id) with Jd[i] */
                gJr[i] += w[i] * s[ir] + w[ir] * s[i];
                gJd[i] += w[i] * s[id] + w[id] * s[i];
            }
        /* passive sites: dL/ds_old(j) = dL/ds_new(j) + sum_i w_i J_ij */
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y) & 1) == colour) continue;
                int j = y * L + x;
                int xl = wrap(x - 1, L), xr = wrap(x + 1, L), yu = wrap(y - 1, L), yd = wrap(y + 1, L);
                g[j] += w[y * L + xr] * Jr[j] + w[y * L + xl] * Jr[y * L + xl]
                      + w[yd * L + x] * Jd[j] + w[yu * L + x] * Jd[yu * L + x];
            }
    }
    free(w);
}

/* L = sum_i (target_i - s_i)^2 (Sec. "Optimization of the exchange       */
/* parameters"); g = dL/ds = -2 (target - s).                             */
double or_dmc_loss(int L, const double *s, const double *target, double *g)
{
    double loss = 0.0;
    for (int i = 0; i < L * L; ++i) {
        double d = target[i] - s[i];
        loss += d * d;
        if (g) g[i] = -2.0 * d;
    }
    return loss;
}

/* Discretisation after the parameter update: s <- -1 if s < 0, else +1. */
void or_dmc_discretize(int n, double *s)
{
    for (int i = 0; i < n; ++i) s[i] = s[i] < 0.0 ? -1.0 : 1.0;
}

/* Energy of relaxed spins under per-bond couplings (Sec. "Optimization of  */
/* the spin values": the loss is the Hamiltonian itself),                   */
/*   E = -sum_<ij> J_ij s_i s_j - h sum_i s_i  (each bond once),            */
/* and g = dE/ds: g_i = -(n_i + h), n_i = sum_j J_ij s_j.                   */
double or_dmc_energy(int L, const double *Jr, const double *Jd, double h, const double *s, double *g)
{
    double E = 0.0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int i = y * L + x;
            E -= Jr[i] * s[i] * s[y * L + wrap(x + 1, L)];
            E -= Jd[i] * s[i] * s[wrap(y + 1, L) * L + x];
            E -= h * s[i];
            if (g) g[i] = -(dmc_field(L, Jr, Jd, s, x, y) + h);
        }
    return E;
}

/* Spin-value step with a quantised gradient (reading of Sec. "Optimization */
/* of the spin values"): s <- clip(s - eta * sign(g), -1, 1), sign(0) = 0.   */
void or_dmc_spin_step(int n, double *s, const double *g, double eta)
{
    for (int i = 0; i < n; ++i) {
        double sg = g[i] > 0.0 ? 1.0 : (g[i] < 0.0 ? -1.0 : 0.0);
        double v = s[i] - eta * sg;
        s[i] = v > 1.0 ? 1.0 : (v < -1.0 ? -1.0 : v);
    }
}

/* ------------------------------------------------------------------ */
/* Ising model on the triangular lattice (Sec. "Ising model": other     */
/* connectivities through a kernel matching the lattice geometry).  The */
/* triangular lattice is stored on the square grid with six neighbours  */
/* (x+-1, y), (x, y+-1), (x+1, y-1), (x-1, y+1), periodic; every bond is */
/* counted once through (x+1, y), (x, y+1), (x-1, y+1).  Three colours   */
/* c = (x - y) mod 3 (no bond joins two sites of one colour; L % 3 == 0) */
/* replace the two of the checkerboard, updated in the order 0, 1, 2.    */
/* The draw of site (x, y) of colour c: k = y (L/3) + (x div 3),         */
/* Philox(seed; k >> 2, lattice, sweep, c), lane k & 3.                  */
/* ------------------------------------------------------------------ */
static int tri_nsum(int L, const int8_t *s, int x, int y)
{
    int xl = wrap(x - 1, L), xr = wrap(x + 1, L), yu = wrap(y - 1, L), yd = wrap(y + 1, L);
    return s[y * L + xl] + s[y * L + xr] + s[yu * L + x] + s[yd * L + x] + s[yu * L + xr] + s[yd * L + xl];
}

void or_tri_substep(int L, float beta, float J, float h, uint64_t seed, uint32_t lattice, uint32_t sweep,
                    int colour, int8_t *s)
{
    double beta_d = (double)beta;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            if (((x - y) % 3 + 3) % 3 != colour) continue;
            int sig = s[y * L + x];
            int n = tri_nsum(L, s, x, y);
            double dE = 2.0 * (double)sig * ((double)J * (double)n + (double)h);
            uint32_t k = (uint32_t)(y * (L / 3) + x / 3);
            uint32_t r[4];
            draw4(seed, k >> 2, lattice, sweep, (uint32_t)colour, r);
            if (or_accept(beta_d, dE, r[k & 3u])) s[y * L + x] = (int8_t)(-sig);
        }
}

void or_tri_sweep(int L, float beta, float J, float h, uint64_t seed, uint32_t lattice, uint32_t sweep, int8_t *s)
{
    for (int c = 0; c < 3; ++c) or_tri_substep(L, beta, J, h, seed, lattice, sweep, c, s);
}

/* out[0] = M = sum s, out[1] = B = sum over bonds of s_i s_j (3 per site). */
void or_tri_stats(int L, const int8_t *s, int64_t out[2])
{
    int64_t M = 0, B = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int v = s[y * L + x];
            M += v;
            B += v * (s[y * L + wrap(x + 1, L)] + s[wrap(y + 1, L) * L + x] + s[wrap(y + 1, L) * L + wrap(x - 1, L)]);
        }
    out[0] = M;
    out[1] = B;
}

void or_tri_run(int L, float beta, float J, float h, uint64_t seed, uint32_t lattice, uint32_t sweep0,
                int nsweeps, int8_t *s, int64_t *stats)
{
    for (int t = 0; t < nsweeps; ++t) {
        or_tri_sweep(L, beta, J, h, seed, lattice, sweep0 + (uint32_t)t, s);
        if (stats) or_tri_stats(L, s, stats + 2 * (size_t)t);
    }
}

/* ------------------------------------------------------------------ */
/* Ising model with first and second neighbours (Sec. "Ising model": the */
/* checkerboard update serves any order of neighbourhood as long as a    */
/* site's colour differs from the colours of all its neighbours).        */
/* H = -J sum_nn s s - J2 sum_nnn s s - h sum s over the four nearest    */
/* neighbours (x+-1, y), (x, y+-1) and the four diagonal ones            */
/* (x+-1, y+-1), periodic; every bond counted once (nearest through      */
/* (x+1, y), (x, y+1); diagonal through (x+1, y+1), (x+1, y-1)).  Four   */
/* colours c = (x & 1) | ((y & 1) << 1), updated in the order 0..3       */
/* (L even).  A flip changes the energy by dE = 2 s (J n1 + J2 n2 + h),  */
/* n1 and n2 the sums of the nearest and of the diagonal neighbours.     */
/* The draw of site (x, y) of colour c: k = (y >> 1)(L/2) + (x >> 1),    */
/* Philox(seed; k >> 2, lattice, sweep, c), lane k & 3.                  */
/* ------------------------------------------------------------------ */
static void nnn_sums(int L, const int8_t *s, int x, int y, int *n1, int *n2)
{
    int xl = wrap(x - 1, L), xr = wrap(x + 1, L), yu = wrap(y - 1, L), yd = wrap(y + 1, L);
    *n1 = s[y * L + xl] + s[y * L + xr] + s[yu * L + x] + s[yd * L + x];
    *n2 = s[yu * L + xl] + s[yu * L + xr] + s[yd * L + xl] + s[yd * L + xr];
}

void or_nnn_substep(int L, float beta, float J, float J2, float h, uint64_t seed, uint32_t lattice,
                    uint32_t sweep, int colour, int8_t *s)
{
    double beta_d = (double)beta;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            if (((x & 1) | ((y & 1) << 1)) != colour) continue;
            int sig = s[y * L + x], n1, n2;
            nnn_sums(L, s, x, y, &n1, &n2);
            double dE = 2.0 * (double)sig * ((double)J * (double)n1 + (double)J2 * (double)n2 + (double)h);
            uint32_t k = (uint32_t)((y >> 1) * (L / 2) + (x >> 1));
            uint32_t r[4];
            draw4(seed, k >> 2, lattice, sweep, (uint32_t)colour, r);
            if (or_accept(beta_d, dE, r[k & 3u])) s[y * L + x] = (int8_t)(-sig);
        }
}

void or_nnn_sweep(int L, float beta, float J, float J2, float h, uint64_t seed, uint32_t lattice,
                  uint32_t sweep, int8_t *s)
{
    for (int c = 0; c < 4; ++c) or_nnn_substep(L, beta, J, J2, h, seed, lattice, sweep, c, s);
}

/* out[0] = M = sum s, out[1] = B = sum over nearest-neighbour bonds of s s,
 * out[2] = B2 = sum over diagonal bonds of s s (two of each per site).      */
void or_nnn_stats(int L, const int8_t *s, int64_t out[3])
{
    int64_t M = 0, B = 0, B2 = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int v = s[y * L + x], xr = wrap(x + 1, L), yd = wrap(y + 1, L), yu = wrap(y - 1, L);
            M += v;
            B += v * (s[y * L + xr] + s[yd * L + x]);
            B2 += v * (s[yd * L + xr] + s[yu * L + xr]);
        }
    out[0] = M;
    out[1] = B;
    out[2] = B2;
}

void or_nnn_run(int L, float beta, float J, float J2, float h, uint64_t seed, uint32_t lattice,
                uint32_t sweep0, int nsweeps, int8_t *s, int64_t *stats)
{
    for (int t = 0; t < nsweeps; ++t) {
        or_nnn_sweep(L, beta, J, J2, h, seed, lattice, sweep0 + (uint32_t)t, s);
        if (stats) or_nnn_stats(L, s, stats + 3 * (size_t)t);
    }
}
