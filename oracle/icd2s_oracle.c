/*
 * icd2s_oracle.c -- plain, slow, single-threaded CPU oracle for the IC-D2S
 * emulated-Ising-machine step (Abdollahi, Kamal, Pedram, "IC-D2S: A Hybrid
 * Ising-Classical-Machines Data-Driven QUBO Solver Method", ASP-DAC'25).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Every function follows the paper's definition or algorithm step by step,
 * in the paper's order and notation, with no blocking, fusion or reordering:
 * gains are recomputed from their definition wherever the paper recomputes
 * them, the subQUBO is built explicitly with its boundary bias (Eq. 4), and
 * the annealer recomputes each local gain from the subQUBO matrix on every
 * attempt.  Integer quantities are exact (int64 energies); the only floating
 * point is in the host tables (cosine temperature schedule, -ln table,
 * mutation-rate schedule), computed in double with the C library.
 *
 * Readings of the paper where it is silent or inconsistent (numbered S1..S24
 * in the design notes) are marked at the place they apply.
 *
 * Pins (tests/test_oracle_*.py): brute force over all 2^n assignments for
 * small n, the closed-form single-flip energy change, the Ising-form identity
 * (Eq. 2-3), hand-worked control-parameter examples, the closed-form values
 * of the mutation-rate schedule (Eq. 5), the Metropolis acceptance
 * probability of the threshold table, and Philox against an independent
 * generator (counter 0, and counter words 0, 1 and 2 at chosen offsets).  The anneal temperatures (T_max, T_min) have no
 * value in the paper: trajectory equality holds for any value, solution
 * quality at a given value is parity unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_TAG_INIT 1u
#define ORC_TAG_ANNEAL 2u
#define ORC_TAG_MUT 3u
#define ORC_TAG_SIZE 4u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator, written from its definition in     */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" */
/* (SC'11): ten rounds of two 32x32->64 multiplies, a Weyl key schedule.     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One 32-bit word of Philox at counter (c0, c1, c2, c3), key = seed halves. */
static uint32_t orc_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                         uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: f(x) = sum_i Q_ii x_i + sum_i sum_{j != i} Q_ij x_i x_j.           */
/* ------------------------------------------------------------------------ */
int64_t orc_energy(const int8_t* Q, int32_t n, const uint8_t* x)
{
    int64_t f = 0;
    for (int32_t i = 0; i < n; ++i)
        f += (int64_t)Q[(int64_t)i * n + i] * x[i];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j)
            if (j != i)
                f += (int64_t)Q[(int64_t)i * n + j] * x[i] * x[j];
    return f;
}

/* 1-flip move value of every variable (Section 2.4, Algorithm 1),
 * with the factor 2 that a symmetric Q needs (reading S1):
 *   g_k = (1 - 2 x_k) (Q_kk + 2 sum_{j != k} Q_jk x_j)
 * which equals f(x with x_k flipped) - f(x). */
void orc_gains(const int8_t* Q, int32_t n, const uint8_t* x, int32_t* g)
{
    for (int32_t k = 0; k < n; ++k) {
        int64_t s = 0;
        for (int32_t j = 0; j < n; ++j)
            if (j != k && x[j])
                s += Q[(int64_t)j * n + k];
        g[k] = (int32_t)((1 - 2 * (int64_t)x[k]) * (Q[(int64_t)k * n + k] + 2 * s));
    }
}

/* Energy of `count` row vectors x[count][n]. */
void orc_energy_batch(const int8_t* Q, int32_t n, const uint8_t* x, int32_t count, int64_t* E)
{
    for (int32_t p = 0; p < count; ++p)
        E[p] = orc_energy(Q, n, x + (int64_t)p * n);
}

/* ------------------------------------------------------------------------ */
/* Host tables.                                                              */
/* ------------------------------------------------------------------------ */

/* Cosine temperature schedule of the emulated Ising machine (reading S13):
 * T_k = T_min + (T_max - T_min) (1 + cos(pi k / (K - 1))) / 2 for K > 1,
 * T_0 = T_min for K = 1;  BETA[k] = round(2^24 / T_k), saturated to uint32. */
void orc_beta_table(int32_t sweeps, double T_max, double T_min, uint32_t* beta)
{
    for (int32_t k = 0; k < sweeps; ++k) {
        double T;
        if (sweeps > 1)
            T = T_min + (T_max - T_min) * (1.0 + cos(M_PI * (double)k / (double)(sweeps - 1))) / 2.0;
        else
            T = T_min;
        double b = 16777216.0 / T;
        if (!(b < 4294967295.0))
            beta[k] = 4294967295u;
        else
            beta[k] = (uint32_t)llround(b);
    }
}

/* -ln table for the fixed-point Metropolis test (reading S14):
 * NLOG[j] = round(2^24 * -ln((j + 0.5) / 4096)), j = 0..4095. */
void orc_nlog_table(uint32_t* nlog)
{
    for (int32_t j = 0; j < 4096; ++j)
        nlog[j] = (uint32_t)llround(16777216.0 * -log(((double)j + 0.5) / 4096.0));
}

/* Eq. 5 (MRAnnealer): r_t = 0.3 (1 + cos(pi t / 15)) 0.99^t. */
double orc_mutation_rate(int32_t t)
{
    return 0.3 * (1.0 + cos(M_PI * (double)t / 15.0)) * pow(0.99, (double)t);
}

/* ------------------------------------------------------------------------ */
/* Generate_Initial_Solution_Set (Algorithm 2): z random binary rows.        */
/* x[p][j] = bit (j mod 32) of word ((j / 32) mod 4) of                      */
/* Philox(ctr = (j / 128, TAG_INIT << 24, p, 0), key = seed).                */
/* ------------------------------------------------------------------------ */
void orc_init_solutions(int32_t n, int32_t z, uint64_t seed, uint8_t* S)
{
    for (int32_t p = 0; p < z; ++p)
        for (int32_t j = 0; j < n; ++j) {
            uint32_t w = orc_word(seed, (uint32_t)(j / 128), ORC_TAG_INIT << 24,
                                  (uint32_t)p, 0u, (j / 32) % 4);
            S[(int64_t)p * n + j] = (uint8_t)((w >> (j % 32)) & 1u);
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Tabu search, Section 2.4) with readings S1-S7:               */
/*  - gains carry the symmetric factor 2 (S1) and the update uses the sign   */
/*    of both variables (S2);                                                */
/*  - OV accumulates the gain of the chosen move before it is negated (S3);  */
/*  - no aspiration (S4); tenure as written: C[i] += c, then every positive  */
/*    C decrements in the same iteration (S5);                               */
/*  - argmin ties go to the lowest index; with 1 <= c <= n some variable is  */
/*    always free (S6);                                                      */
/*  - C and T start at zero on every call and the call returns x_min (S7).   */
/* x is replaced by x_min; T (toggle counts) and C (tabu memory at the end)  */
/* are returned; the return value is OV_min = f(x_min).                      */
/* ------------------------------------------------------------------------ */
int64_t orc_tabu_asp(const int8_t* Q, int32_t n, uint8_t* x, int32_t alpha, int32_t c,
                     int32_t* T, int32_t* C, int32_t aspiration, int32_t* moves);
int64_t orc_tabu(const int8_t* Q, int32_t n, uint8_t* x, int32_t alpha, int32_t c,
                 int32_t* T, int32_t* C)
{
    return orc_tabu_asp(Q, n, x, alpha, c, T, C, 0, NULL);
}

/* The same search with the aspiration criterion the text of Section 2.4
 * describes (reading S4: off by default): a tabu move is admissible when it
 * would give a better objective than the best visited so far.  A variable
 * moved while tabu adds c to its remaining tabu memory, so with aspiration
 * every move can become tabu; the search then takes the unmasked arg-min
 * (reading S6).  moves[alpha] (optional) receives the variable moved at each
 * iteration. */
int64_t orc_tabu_asp(const int8_t* Q, int32_t n, uint8_t* x, int32_t alpha, int32_t c,
                     int32_t* T, int32_t* C, int32_t aspiration, int32_t* moves)
{
    int32_t* dx = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t* xmin = (uint8_t*)malloc((size_t)n);
    int64_t OV = orc_energy(Q, n, x);                  /* objective value */
    int64_t OVmin = OV;
    memcpy(xmin, x, (size_t)n);
    orc_gains(Q, n, x, dx);                            /* all 1-flip move values */
    for (int32_t k = 0; k < n; ++k) { C[k] = 0; T[k] = 0; }
    for (int32_t it = 0; it < alpha; ++it) {
        int32_t i = -1;                                /* argmin over the non-tabu moves (C <= 0) */
        for (int32_t k = 0; k < n; ++k) {
            const int admissible = C[k] <= 0 || (aspiration && OV + dx[k] < OVmin);
            if (admissible && (i < 0 || dx[k] < dx[i]))
                i = k;
        }
        if (i < 0)                                     /* every move tabu, none aspirated */
            for (int32_t k = 0; k < n; ++k)
                if (i < 0 || dx[k] < dx[i])
                    i = k;
        if (moves) moves[it] = i;
        int32_t gi = dx[i];
        int32_t si = 1 - 2 * x[i];
        for (int32_t j = 0; j < n; ++j)                /* O(n) move-value update */
            if (j != i)
                dx[j] += 2 * Q[(int64_t)i * n + j] * si * (1 - 2 * x[j]);
        dx[i] = -gi;
        OV += gi;
        C[i] += c;
        x[i] = (uint8_t)(1 - x[i]);
        T[i] += 1;                                     /* toggle count (Eq. 7) */
        for (int32_t k = 0; k < n; ++k)                /* tabu memory decays */
            if (C[k] > 0)
                C[k] -= 1;
        if (OV < OVmin) {                              /* keep the best visited */
            memcpy(xmin, x, (size_t)n);
            OVmin = OV;
        }
    }
    memcpy(x, xmin, (size_t)n);                        /* the search returns x_min */
    free(dx);
    free(xmin);
    return OVmin;
}

/* ------------------------------------------------------------------------ */
/* Control parameters (Section 3).                                           */
/* ------------------------------------------------------------------------ */

/* Eq. 6: eta_j = sum_i |Q_ij|. */
void orc_eta(const int8_t* Q, int32_t n, int64_t* eta)
{
    for (int32_t j = 0; j < n; ++j) {
        int64_t s = 0;
        for (int32_t i = 0; i < n; ++i)
            s += llabs((long long)Q[(int64_t)i * n + j]);
        eta[j] = s;
    }
}

/* Reading S9: eta is normalised by its maximum so that it is on the same
 * [0, 1] scale as gamma and Delta; Q16 fixed point, floor. */
void orc_eta_hat(const int64_t* eta, int32_t n, int32_t* eta_hat)
{
    int64_t mx = 0;
    for (int32_t j = 0; j < n; ++j)
        if (eta[j] > mx) mx = eta[j];
    for (int32_t j = 0; j < n; ++j)
        eta_hat[j] = mx > 0 ? (int32_t)((eta[j] * 65536) / mx) : 0;
}

/* Eq. 8: gamma_j = 1 - |sum_i S_ij - z/2| / (z/2) = (z - |2 sum_i S_ij - z|) / z,
 * Q16 fixed point, floor. */
void orc_gamma(const uint8_t* S, int32_t z, int32_t n, int32_t* gamma)
{
    for (int32_t j = 0; j < n; ++j) {
        int64_t col = 0;
        for (int32_t p = 0; p < z; ++p)
            col += S[(int64_t)p * n + j];
        int64_t dev = 2 * col - z;
        if (dev < 0) dev = -dev;
        gamma[j] = (int32_t)(((int64_t)z - dev) * 65536 / z);
    }
}

/* Eq. 7: Delta_pj = 1 - T_pj / max_j T_pj, Q16 fixed point, floor;
 * Delta = 0 when no variable toggled. */
void orc_delta(const int32_t* T, int32_t n, int32_t* delta)
{
    int64_t mx = 0;
    for (int32_t j = 0; j < n; ++j)
        if (T[j] > mx) mx = T[j];
    for (int32_t j = 0; j < n; ++j)
        delta[j] = mx > 0 ? (int32_t)((mx - T[j]) * 65536 / mx) : 0;
}

static int64_t orc_floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b, r = a % b;
    if (r != 0 && ((r < 0) != (b < 0))) q -= 1;
    return q;
}

/* Algorithm 3 (Control_Parameters_Aggregation), one row:
 * A_j = w1 eta_j + w2 gamma_j - w3 Delta_j, with Q16 weights and Q16
 * parameters; the Q32 product is floored back to Q16. */
void orc_aggregate(const int32_t* eta_hat, const int32_t* gamma, const int32_t* delta,
                   int32_t n, int64_t w1, int64_t w2, int64_t w3, int32_t* A)
{
    for (int32_t j = 0; j < n; ++j) {
        int64_t v = w1 * eta_hat[j] + w2 * gamma[j] - w3 * delta[j];
        A[j] = (int32_t)orc_floor_div(v, 65536);
    }
}

/* ------------------------------------------------------------------------ */
/* Selection (Algorithm 4, choice of S').  Rank variables by (A desc, index  */
/* asc); the first sum_k m_k ranks are S'; group k takes ranks               */
/* [m_0 + .. + m_{k-1}, m_0 + .. + m_k) (one subQUBO per Ising machine,      */
/* reading S16); each group is listed in ascending index order (S15).        */
/* ------------------------------------------------------------------------ */
static const int32_t* orc_sort_key;
static int orc_cmp_rank(const void* a, const void* b)
{
    int32_t i = *(const int32_t*)a, j = *(const int32_t*)b;
    if (orc_sort_key[i] != orc_sort_key[j])
        return orc_sort_key[i] > orc_sort_key[j] ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}
static int orc_cmp_int(const void* a, const void* b)
{
    int32_t i = *(const int32_t*)a, j = *(const int32_t*)b;
    return i < j ? -1 : (i > j ? 1 : 0);
}

/* order[n] := variables ranked by (key desc, index asc). */
void orc_rank(const int32_t* key, int32_t n, int32_t* order)
{
    for (int32_t j = 0; j < n; ++j) order[j] = j;
    orc_sort_key = key;
    qsort(order, (size_t)n, sizeof(int32_t), orc_cmp_rank);
}

/* idx[sum sizes] receives the K groups back to back. */
void orc_select(const int32_t* A, int32_t n, const int32_t* sizes, int32_t K, int32_t* idx)
{
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    orc_rank(A, n, order);
    int32_t off = 0;
    for (int32_t k = 0; k < K; ++k) {
        memcpy(idx + off, order + off, sizeof(int32_t) * (size_t)sizes[k]);
        qsort(idx + off, (size_t)sizes[k], sizeof(int32_t), orc_cmp_int);
        off += sizes[k];
    }
    free(order);
}

/* Uneven subQUBO sizes of one replica at one iteration (reading S18):
 * m_k = m_min + (Philox(ctr = (k, TAG_SIZE << 24, p, iter)).word0 mod (m_max - m_min + 1)). */
void orc_subqubo_sizes(int32_t K, int32_t m_min, int32_t m_max, uint64_t seed, uint32_t p,
                       uint32_t iter, int32_t* sizes)
{
    for (int32_t k = 0; k < K; ++k) {
        if (m_max == m_min) { sizes[k] = m_min; continue; }
        uint32_t u = orc_word(seed, (uint32_t)k, ORC_TAG_SIZE << 24, p, iter, 0);
        sizes[k] = m_min + (int32_t)(u % (uint32_t)(m_max - m_min + 1));
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 4 / Algorithm 4: the subQUBO Q' of the variables S (m of them), with */
/* the boundary bias b_i = sum_{j not in S} 2 Q_ij x_j added on its          */
/* diagonal.  The pair sum of Eq. 4 is read over i != j (S8).                */
/* Qs is m x m int32; b (optional) receives the bias.                       */
/* ------------------------------------------------------------------------ */
void orc_subqubo(const int8_t* Q, int32_t n, const uint8_t* x, const int32_t* S, int32_t m,
                 int32_t* Qs, int64_t* b_out)
{
    uint8_t* in_s = (uint8_t*)calloc((size_t)n, 1);
    for (int32_t a = 0; a < m; ++a) in_s[S[a]] = 1;
    for (int32_t a = 0; a < m; ++a) {
        int64_t b = 0;
        for (int32_t j = 0; j < n; ++j)
            if (!in_s[j])
                b += 2 * (int64_t)Q[(int64_t)S[a] * n + j] * x[j];
        for (int32_t c = 0; c < m; ++c)
            Qs[(int64_t)a * m + c] = Q[(int64_t)S[a] * n + S[c]];
        Qs[(int64_t)a * m + a] = (int32_t)(Q[(int64_t)S[a] * n + S[a]] + b);
        if (b_out) b_out[a] = b;
    }
    free(in_s);
}

/* Exact Ising machine for small subQUBOs (the "precise solution" of a
 * subQUBO, Section 3): the assignment y of the m positions that minimises
 * the Eq. 4 objective, found by trying all 2^m of them; ties go to the
 * smallest y read as the integer sum_a y_a 2^a.  xs[m] is replaced by the
 * minimiser; returns f(y) - f(xs).  m <= 24. */
int64_t orc_subqubo_energy(const int32_t* Qs, int32_t m, const uint8_t* xs);
int64_t orc_exact_subqubo(const int32_t* Qs, int32_t m, uint8_t* xs)
{
    uint8_t* y = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
    const int64_t f0 = orc_subqubo_energy(Qs, m, xs);
    int64_t best = INT64_MAX;
    uint32_t best_v = 0;
    for (uint32_t v = 0; v < (1u << m); ++v) {
        for (int32_t a = 0; a < m; ++a) y[a] = (uint8_t)((v >> a) & 1u);
        const int64_t f = orc_subqubo_energy(Qs, m, y);
        if (f < best) { best = f; best_v = v; }
    }
    for (int32_t a = 0; a < m; ++a) xs[a] = (uint8_t)((best_v >> a) & 1u);
    free(y);
    return best - f0;
}

/* Energy of the subQUBO (Eq. 4 objective) at xs[m]. */
int64_t orc_subqubo_energy(const int32_t* Qs, int32_t m, const uint8_t* xs)
{
    int64_t f = 0;
    for (int32_t a = 0; a < m; ++a)
        f += (int64_t)Qs[(int64_t)a * m + a] * xs[a];
    for (int32_t a = 0; a < m; ++a)
        for (int32_t c = 0; c < m; ++c)
            if (c != a)
                f += (int64_t)Qs[(int64_t)a * m + c] * xs[a] * xs[c];
    return f;
}

/* ------------------------------------------------------------------------ */
/* Emulated Ising machine (Algorithm 4, solve step; readings S13-S15):      */
/* single-flip Metropolis annealing of the subQUBO Qs at xs, `sweeps`        */
/* sweeps over positions 0..m-1 in order, sweep k at inverse temperature     */
/* BETA[k] (Q24).  Attempt (k, pos) draws                                    */
/*   u = Philox(ctr = (k / 4, (TAG_ANNEAL << 24) | pos, slot, iter)).word[k mod 4]
 * and accepts iff the local gain l <= 0 or l * BETA[k] < NLOG[u >> 20].     */
/* The local gain is recomputed from Qs on every attempt.                    */
/* Returns the subQUBO energy change; *accepts counts accepted flips.        */
/* ------------------------------------------------------------------------ */
int64_t orc_anneal(const int32_t* Qs, int32_t m, uint8_t* xs, int32_t sweeps,
                   const uint32_t* beta, const uint32_t* nlog, uint64_t seed,
                   uint32_t slot, uint32_t iter, int64_t* accepts)
{
    int64_t dE = 0, acc = 0;
    for (int32_t k = 0; k < sweeps; ++k) {
        for (int32_t pos = 0; pos < m; ++pos) {
            int64_t field = Qs[(int64_t)pos * m + pos];
            for (int32_t c = 0; c < m; ++c)
                if (c != pos)
                    field += 2 * (int64_t)Qs[(int64_t)pos * m + c] * xs[c];
            int64_t l = (1 - 2 * (int64_t)xs[pos]) * field;
            uint32_t u = orc_word(seed, (uint32_t)(k / 4), (ORC_TAG_ANNEAL << 24) | (uint32_t)pos,
                                  slot, iter, k % 4);
            int accept = (l <= 0) || ((uint64_t)l * (uint64_t)beta[k] < (uint64_t)nlog[u >> 20]);
            if (accept) {
                xs[pos] = (uint8_t)(1 - xs[pos]);
                dE += l;
                acc += 1;
            }
        }
    }
    if (accepts) *accepts = acc;
    return dE;
}

/* ------------------------------------------------------------------------ */
/* Mutation (Section 3, end; readings S10, S11): the L variables outside S'  */
/* with the highest A (index ascending on ties) are candidates; candidate i  */
/* flips iff Philox(ctr = (i / 4, TAG_MUT << 24, p, iter)).word[i mod 4] <   */
/* P_i with P_i = floor((A_i - A_min)(2^32 - 1) / (A_max - A_min)) over the  */
/* whole row (2^31 when A_max = A_min).  Returns the number of flips.        */
/* ------------------------------------------------------------------------ */
static int32_t orc_mutate_p(const int32_t* A, int32_t n, const uint8_t* in_sel, int32_t L, uint64_t seed,
                            uint32_t p, uint32_t iter, uint8_t* x, int half);
int32_t orc_mutate(const int32_t* A, int32_t n, const uint8_t* in_sel, int32_t L, uint64_t seed,
                   uint32_t p, uint32_t iter, uint8_t* x)
{
    return orc_mutate_p(A, n, in_sel, L, seed, p, iter, x, 0);
}

/* half != 0: every candidate flips with probability 1/2 (P = 2^31), the
 * No_SM ablation's mutation without control parameters. */
static int32_t orc_mutate_p(const int32_t* A, int32_t n, const uint8_t* in_sel, int32_t L, uint64_t seed,
                            uint32_t p, uint32_t iter, uint8_t* x, int half)
{
    int32_t amin = A[0], amax = A[0];
    for (int32_t j = 1; j < n; ++j) {
        if (A[j] < amin) amin = A[j];
        if (A[j] > amax) amax = A[j];
    }
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    orc_rank(A, n, order);
    int32_t taken = 0, flips = 0;
    for (int32_t r = 0; r < n && taken < L; ++r) {
        int32_t i = order[r];
        if (in_sel[i]) continue;
        taken += 1;
        uint64_t P;
        if (amax == amin || half)
            P = 2147483648ull;
        else
            P = ((uint64_t)((int64_t)A[i] - amin) * 4294967295ull) / (uint64_t)((int64_t)amax - amin);
        uint32_t u = orc_word(seed, (uint32_t)(i / 4), ORC_TAG_MUT << 24, p, iter, i % 4);
        if ((uint64_t)u < P) {
            x[i] = (uint8_t)(1 - x[i]);
            flips += 1;
        }
    }
    free(order);
    return flips;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: the whole IC-D2S loop.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t z;          /* solutions (replicas) */
    int32_t K;          /* subQUBOs per solution per call (multi-IM fabric) */
    int32_t m_min, m_max; /* subQUBO size range (equal for the plain method) */
    int32_t m_init;     /* block size of Call_IM_Solution_Set */
    int32_t alpha;      /* Tabu iterations */
    int32_t c;          /* Tabu tenure increment */
    int32_t sweeps;     /* anneal sweeps per subQUBO */
    double T_max, T_min;
    int64_t w1, w2, w3; /* Q16 aggregation weights */
    int32_t mut_mode;   /* 0: Eq. 5 schedule r_t; 1: constant rate */
    double mut_rate;
    int32_t patience;   /* stop after this many iterations without a new best (<= 0: off) */
    int32_t max_iters;
    int32_t select_mode; /* 0: rank by A (Algorithm 4); 1: rank by the learned score;
                            2: learned on even solutions, A on odd ones */
    int32_t im_mode;     /* 0: annealing Ising machine; 1: exact (m_max <= 24) */
    int32_t ablation;    /* 0: the method; 1: No_IM (no Ising-machine call); 2: No_SM (no control
                            parameters: a random ranking and flip probability 1/2) */
    int32_t aspiration;  /* Tabu search with the aspiration criterion (reading S4) */
    int32_t im_order;    /* K > 1 subQUBOs of a solution: 0 = every one built from the state before
                            the call (Jacobi merge, reading S16); 1 = one after the other, each built
                            from the state the previous ones left (Gauss-Seidel, the order in which
                            Section 3 describes Call_IM_Solution_Set) */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Learned selection (the added proposal network; readings S21, S22).        */
/* ------------------------------------------------------------------------ */

/* Per-variable features of one solution at selection time, as floats:
 *   f0 = x_i, f1 = g_i / (max_j |g_j| + 1), f2 = T_i / alpha, f3 = C_i / c,
 *   f4 = H_i / (t + 1), f5 = eta_hat_i / 2^16,
 * with g the 1-flip gains, T and C the toggle counts and tabu memory of the
 * last Tabu search, H the number of earlier Ising-machine calls that included
 * the variable and t the outer iteration.  Every quotient is of two integers
 * below 2^24 (exact in float); it is formed in double and rounded once to
 * float, which gives the correctly rounded float quotient because double
 * has more than 2 * 24 + 2 significand bits.  alpha = 0 gives f2 = 0. */
void orc_features(int32_t n, const uint8_t* x, const int32_t* g, const int32_t* T, const int32_t* C,
                  const int32_t* H, const int32_t* eta_hat, int32_t t, int32_t alpha, int32_t c, float* F)
{
    int64_t gmax = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = g[i] < 0 ? -(int64_t)g[i] : g[i];
        if (a > gmax) gmax = a;
    }
    for (int32_t i = 0; i < n; ++i) {
        float* f = F + (int64_t)i * 6;
        f[0] = (float)x[i];
        f[1] = (float)((double)g[i] / (double)(gmax + 1));
        f[2] = alpha > 0 ? (float)((double)T[i] / (double)alpha) : 0.0f;
        f[3] = (float)((double)C[i] / (double)c);
        f[4] = (float)((double)H[i] / (double)(t + 1));
        f[5] = (float)((double)eta_hat[i] / 65536.0);
    }
}

/* Parameter layout of the 6-64-64-1 network (4673 values): W1[64][6], b1[64],
 * W2[64][64], b2[64], w3[64], b3.  Row o of W1/W2 holds the weights into
 * hidden unit o. */
#define ORC_W1 0
#define ORC_B1 384
#define ORC_W2 448
#define ORC_B2 4544
#define ORC_W3 4608
#define ORC_B3 4672
#define ORC_NPAR 4673

/* Score of one feature row in float arithmetic, the precision in which the
 * selection decision is taken: ReLU hidden layers, every product added by
 * one fused multiply-add (fmaf), units and inputs in increasing order:
 *   a1_o = b1_o (+ W1_o0 f_0) ... (+ W1_o5 f_5),        h1_o = max(a1_o, 0)
 *   a2_o = b2_o (+ W2_o0 h1_0) ... (+ W2_o63 h1_63),    h2_o = max(a2_o, 0)
 *   s    = b3 (+ w3_0 h2_0) ... (+ w3_63 h2_63).
 * W holds BF16 values widened to float. */
float orc_mlp_score_f32(const float* W, const float* f)
{
    float h1[64];
    for (int o = 0; o < 64; ++o) {
        float a = W[ORC_B1 + o];
        for (int k = 0; k < 6; ++k) a = fmaf(W[ORC_W1 + o * 6 + k], f[k], a);
        h1[o] = a > 0.0f ? a : 0.0f;
    }
    float s = W[ORC_B3];
    for (int o = 0; o < 64; ++o) {
        float a = W[ORC_B2 + o];
        for (int k = 0; k < 64; ++k) a = fmaf(W[ORC_W2 + o * 64 + k], h1[k], a);
        float h2 = a > 0.0f ? a : 0.0f;
        s = fmaf(W[ORC_W3 + o], h2, s);
    }
    return s;
}

/* A signed integer with the order of the float s (a total order on the bit
 * patterns: -0 ranks just below +0), so that ranking by (score desc, index
 * asc) is the same integer ranking as for A. */
int32_t orc_score_key(float s)
{
    uint32_t b;
    memcpy(&b, &s, 4);
    if (b < 0x80000000u) return (int32_t)b;
    return -(int32_t)(b & 0x7FFFFFFFu) - 1;
}

typedef struct {
    int32_t iters;            /* outer iterations run */
    int64_t best_E;
    int64_t init_best_E;      /* best after Call_IM_Solution_Set */
} orc_result;

static void orc_best_update(const uint8_t* S, const int64_t* E, int32_t z, int32_t n,
                            int64_t* best_E, uint8_t* best_x, int* improved, int32_t* winner)
{
    for (int32_t p = 0; p < z; ++p)
        if (E[p] < *best_E) {
            *best_E = E[p];
            memcpy(best_x, S + (int64_t)p * n, (size_t)n);
            *improved = 1;
            if (winner) *winner = p;
        }
}

/* One outer iteration t of Algorithm 2 on the solution set S[z][n], in
 * place: Tabu search (Algorithm 1), Deviation_Extraction (Eq. 8),
 * Control_Parameters_Aggregation (Algorithm 3), Call_IM_Partial_Solution_Set
 * (Algorithm 4) and the mutation with rate r_t (Eq. 5) or a constant rate.
 * E[z] receives the energies after the iteration; trace3[3 z] (optional) the
 * energies after the Tabu search, the Ising-machine step and the mutation;
 * the best solution is folded in after each of the three phases.  T_out,
 * A_out and C_out (optional, z * n) receive the toggle counts, A and the
 * tabu memory at the end of each search; H_io (optional, z * n) counts, per
 * solution and variable, the Ising-machine calls that included it (each
 * selection adds 1).
 * Learned selection (select_mode 1, or 2 on even solutions): the subset S' is
 * ranked by (score desc, index asc) instead of (A desc, index asc), the score
 * being orc_mlp_score_f32 with the network W of the features at selection
 * time (after the Tabu search; H before this iteration's increments); A still
 * ranks the mutation candidates.  H_io is required in that mode.  F_out
 * (z * n * 6) and score_out (z * n, needs W) receive the features and scores
 * of every solution at selection time; *winner (optional) the solution whose
 * row was last copied into best_x in this iteration (-1 if none).
 * Returns 1 if the best energy improved. */
int32_t orc_step(const int8_t* Q, int32_t n, const orc_params* prm, uint64_t seed, int32_t t,
                 const int32_t* eta_hat, uint8_t* S, int64_t* E, int64_t* trace3, int64_t* best_E,
                 uint8_t* best_x, int32_t* T_out, int32_t* A_out, int32_t* C_out, int32_t* H_io,
                 const float* W, float* F_out, float* score_out, int32_t* winner)
{
    const int32_t z = prm->z, K = prm->K;
    if (winner) *winner = -1;
    if (prm->select_mode != 0 && (W == NULL || H_io == NULL)) return -1;
    int32_t* T = (int32_t*)malloc(sizeof(int32_t) * (size_t)z * n);
    int32_t* C = (int32_t*)malloc(sizeof(int32_t) * (size_t)z * n);
    int32_t* A = (int32_t*)malloc(sizeof(int32_t) * (size_t)z * n);
    int32_t* gam = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* del = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* Qs = (int32_t*)malloc(sizeof(int32_t) * (size_t)prm->m_max * prm->m_max);
    uint8_t* xs = (uint8_t*)malloc((size_t)prm->m_max);
    int32_t* sizes = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)K * prm->m_max);
    uint8_t* S_pre = (uint8_t*)malloc((size_t)n);
    uint8_t* in_sel = (uint8_t*)malloc((size_t)z * n);   /* S' of every solution */
    int32_t* msel = (int32_t*)malloc(sizeof(int32_t) * (size_t)z);
    uint32_t* beta = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(prm->sweeps > 0 ? prm->sweeps : 1));
    uint32_t nlog[4096];
    int32_t* g = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    float* F = (float*)malloc(sizeof(float) * (size_t)n * 6);
    int32_t* skey = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int improved = 0;
    orc_beta_table(prm->sweeps, prm->T_max, prm->T_min, beta);
    orc_nlog_table(nlog);

    /* Tabu search on every solution (Algorithm 1) */
    for (int32_t p = 0; p < z; ++p)
        E[p] = orc_tabu_asp(Q, n, S + (int64_t)p * n, prm->alpha, prm->c, T + (int64_t)p * n,
                            C + (int64_t)p * n, prm->aspiration, NULL);
    orc_best_update(S, E, z, n, best_E, best_x, &improved, winner);
    if (trace3) memcpy(trace3, E, sizeof(int64_t) * (size_t)z);
    /* Deviation_Extraction (Eq. 8), Control_Parameters_Aggregation (Algorithm 3) */
    orc_gamma(S, z, n, gam);
    for (int32_t p = 0; p < z; ++p) {
        orc_delta(T + (int64_t)p * n, n, del);
        orc_aggregate(eta_hat, gam, del, n, prm->w1, prm->w2, prm->w3, A + (int64_t)p * n);
        if (prm->ablation == 2)  /* No_SM: the ranking key is Philox(ctr = (j / 4, 7 << 24, p, t)) >> 1 */
            for (int32_t j = 0; j < n; ++j)
                A[(int64_t)p * n + j] =
                    (int32_t)(orc_word(seed, (uint32_t)(j / 4), 7u << 24, (uint32_t)p, (uint32_t)t, j % 4) >> 1);
    }
    /* Call_IM_Partial_Solution_Set (Algorithm 4) */
    for (int32_t p = 0; p < z; ++p) {
        uint8_t* x = S + (int64_t)p * n;
        const int32_t* Ap = A + (int64_t)p * n;
        if (prm->ablation == 1) {  /* No_IM: no subset, no Ising-machine call */
            memset(in_sel + (int64_t)p * n, 0, (size_t)n);
            msel[p] = 0;
            E[p] = orc_energy(Q, n, x);
            continue;
        }
        orc_subqubo_sizes(K, prm->m_min, prm->m_max, seed, (uint32_t)p, (uint32_t)t, sizes);
        const int learned = prm->select_mode == 1 || (prm->select_mode == 2 && p % 2 == 0);
        if (learned || F_out || score_out) {
            orc_gains(Q, n, x, g);
            int32_t* Hp = H_io ? H_io + (int64_t)p * n : NULL;
            if (!Hp) { Hp = skey; memset(Hp, 0, sizeof(int32_t) * (size_t)n); }
            orc_features(n, x, g, T + (int64_t)p * n, C + (int64_t)p * n, Hp, eta_hat, t, prm->alpha,
                         prm->c, F);
            if (F_out) memcpy(F_out + (int64_t)p * n * 6, F, sizeof(float) * (size_t)n * 6);
        }
        if (learned || (score_out && W)) {
            for (int32_t i = 0; i < n; ++i) {
                float s = orc_mlp_score_f32(W, F + (int64_t)i * 6);
                if (score_out) score_out[(int64_t)p * n + i] = s;
                skey[i] = orc_score_key(s);
            }
        }
        orc_select(learned ? skey : Ap, n, sizes, K, idx);
        memcpy(S_pre, x, (size_t)n);
        memset(in_sel + (int64_t)p * n, 0, (size_t)n);
        int32_t off = 0;
        msel[p] = 0;
        for (int32_t k = 0; k < K; ++k) {
            int32_t m = sizes[k];
            /* Jacobi (reading S16): every subQUBO of this call is built
             * from the state before the call; Gauss-Seidel: from the state
             * with the earlier subQUBOs' results written back */
            const uint8_t* base = prm->im_order == 1 ? x : S_pre;
            orc_subqubo(Q, n, base, idx + off, m, Qs, NULL);
            for (int32_t a = 0; a < m; ++a) xs[a] = base[idx[off + a]];
            if (prm->im_mode == 1)
                orc_exact_subqubo(Qs, m, xs);
            else
                orc_anneal(Qs, m, xs, prm->sweeps, beta, nlog, seed, (uint32_t)(p * K + k), (uint32_t)t, NULL);
            for (int32_t a = 0; a < m; ++a) {
                x[idx[off + a]] = xs[a];
                in_sel[(int64_t)p * n + idx[off + a]] = 1;
                if (H_io) H_io[(int64_t)p * n + idx[off + a]] += 1;
            }
            off += m;
            msel[p] += m;
        }
        E[p] = orc_energy(Q, n, x);
    }
    orc_best_update(S, E, z, n, best_E, best_x, &improved, winner);
    if (trace3) memcpy(trace3 + z, E, sizeof(int64_t) * (size_t)z);
    /* Mutation with the MRAnnealer rate (Eq. 5) */
    double r = prm->mut_mode == 0 ? orc_mutation_rate(t) : prm->mut_rate;
    for (int32_t p = 0; p < z; ++p) {
        uint8_t* x = S + (int64_t)p * n;
        int32_t L = (int32_t)floor((double)(n - msel[p]) * r);
        orc_mutate_p(A + (int64_t)p * n, n, in_sel + (int64_t)p * n, L, seed, (uint32_t)p, (uint32_t)t, x,
                     prm->ablation == 2);
        E[p] = orc_energy(Q, n, x);
    }
    orc_best_update(S, E, z, n, best_E, best_x, &improved, winner);
    if (trace3) memcpy(trace3 + 2 * z, E, sizeof(int64_t) * (size_t)z);
    if (T_out) memcpy(T_out, T, sizeof(int32_t) * (size_t)z * n);
    if (A_out) memcpy(A_out, A, sizeof(int32_t) * (size_t)z * n);
    if (C_out) memcpy(C_out, C, sizeof(int32_t) * (size_t)z * n);
    free(T); free(C); free(A); free(gam); free(del); free(Qs); free(xs); free(sizes); free(idx);
    free(S_pre); free(in_sel); free(msel); free(beta);
    free(g); free(F); free(skey);
    return improved;
}

/* Call_IM_Solution_Set (Algorithm 2): floor(n / m) disjoint blocks of m
 * consecutive variables per solution, each solved with the bias of the
 * current values of the others and written back before the next block
 * (Gauss-Seidel).  With K > 1 Ising machines per solution and the Jacobi
 * order (im_order 0), K consecutive blocks are solved at once (reading S24:
 * Section 3 notes that several IMs address several subQUBOs concurrently):
 * each block of a group is built from the solution before the group, and the
 * group's results are written back together.  E[z] receives the energies. */
void orc_initial_pass(const int8_t* Q, int32_t n, const orc_params* prm, uint64_t seed, uint8_t* S, int64_t* E)
{
    const int32_t m = prm->m_init;
    const int32_t G = (prm->K > 1 && prm->im_order == 0) ? prm->K : 1;  /* blocks solved at once */
    int32_t* Qs = (int32_t*)malloc(sizeof(int32_t) * (size_t)m * m);
    uint8_t* xs = (uint8_t*)malloc((size_t)m);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    uint8_t* pre = (uint8_t*)malloc((size_t)n);
    uint32_t* beta = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(prm->sweeps > 0 ? prm->sweeps : 1));
    uint32_t nlog[4096];
    orc_beta_table(prm->sweeps, prm->T_max, prm->T_min, beta);
    orc_nlog_table(nlog);
    const int32_t nb = prm->ablation == 1 ? 0 : n / m;  /* No_IM: no IM call at all */
    for (int32_t p = 0; p < prm->z; ++p) {
        uint8_t* x = S + (int64_t)p * n;
        for (int32_t l0 = 0; l0 < nb; l0 += G) {
            memcpy(pre, x, (size_t)n);  /* the solution before the group */
            for (int32_t l = l0; l < l0 + G && l < nb; ++l) {
                for (int32_t a = 0; a < m; ++a) idx[a] = l * m + a;
                orc_subqubo(Q, n, pre, idx, m, Qs, NULL);
                for (int32_t a = 0; a < m; ++a) xs[a] = pre[idx[a]];
                if (prm->im_mode == 1)
                    orc_exact_subqubo(Qs, m, xs);
                else
                    orc_anneal(Qs, m, xs, prm->sweeps, beta, nlog, seed, (uint32_t)p, 0x80000000u | (uint32_t)l,
                               NULL);
                for (int32_t a = 0; a < m; ++a) x[idx[a]] = xs[a];
            }
        }
        E[p] = orc_energy(Q, n, x);
    }
    free(Qs); free(xs); free(idx); free(pre); free(beta);
}

/* Runs Algorithm 2 from Generate_Initial_Solution_Set.  Outputs: best_x[n],
 * S_out[z][n] (final solutions), trace[max_iters][3 z + 1] (int64,
 * optional): per iteration the energies of all solutions after the Tabu
 * search, after the IM step, after the mutation, then the best energy;
 * init_E[z] (optional): energies after Call_IM_Solution_Set.  Plain
 * selection only (select_mode 0; otherwise returns -1). */
int32_t orc_run(const int8_t* Q, int32_t n, const orc_params* prm, uint64_t seed,
                uint8_t* best_x, uint8_t* S_out, int64_t* trace, int64_t* init_E,
                orc_result* res)
{
    const int32_t z = prm->z;
    if (prm->select_mode != 0) return -1;
    uint8_t* S = (uint8_t*)malloc((size_t)z * n);
    int64_t* E = (int64_t*)malloc(sizeof(int64_t) * (size_t)z);
    int64_t* eta = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* eta_hat = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t best_E = INT64_MAX;
    int improved = 0;

    orc_init_solutions(n, z, seed, S);                 /* Generate_Initial_Solution_Set */
    orc_initial_pass(Q, n, prm, seed, S, E);           /* Call_IM_Solution_Set */
    orc_best_update(S, E, z, n, &best_E, best_x, &improved, NULL);
    if (init_E) memcpy(init_E, E, sizeof(int64_t) * (size_t)z);
    if (res) res->init_best_E = best_E;
    orc_eta(Q, n, eta);                                /* Weight_Effect_Extraction (Eq. 6) */
    orc_eta_hat(eta, n, eta_hat);

    int32_t t = 0, stale = 0;
    while (t < prm->max_iters && (prm->patience <= 0 || stale < prm->patience)) {
        int64_t* tr = trace ? trace + (int64_t)t * (3 * z + 1) : NULL;
        improved = orc_step(Q, n, prm, seed, t, eta_hat, S, E, tr, &best_E, best_x, NULL, NULL, NULL, NULL,
                            NULL, NULL, NULL, NULL);
        if (tr) tr[3 * z] = best_E;
        /* MRAnnealer.NextRate is r_{t+1}; termination rule (Section 3, end) */
        stale = improved ? 0 : stale + 1;
        t += 1;
    }
    if (S_out) memcpy(S_out, S, (size_t)z * n);
    if (res) { res->iters = t; res->best_E = best_E; }
    free(S); free(E); free(eta); free(eta_hat);
    return t;
}
