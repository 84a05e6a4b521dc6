/*
 * wl_oracle.c -- plain, slow CPU oracle for the micromagnetic-ensemble
 * Wang-Landau method (B. D. Stosic, "Parallelizing Wang-Landau algorithm in
 * the field: the micromagnetic ensemble", arXiv:1302.2320).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the GPU library, and it includes nothing
 * from it.
 *
 * Contents (each function names the passage it follows):
 *   - periodic lattices: square, triangular, simple cubic  (the model, Eq. 1),
 *     and the square lattice with open boundaries (Fig. 2)
 *   - Philox4x32-10 counter-based generator (Salmon et al., SC'11), written
 *     from its published definition; the walk's random numbers come from it
 *   - the 4096-entry fixed-point exp threshold table
 *   - one Wang-Landau walk on one micromagnetic line (Eq. 3, Eq. 4 and the
 *     surrounding text: lists, spin-exchange move, g/h update, flatness,
 *     f -> f^(1/4), stop at f_min), with the optional extra histogram reset
 *     at unchanged f (the remark after Eq. 4)
 *   - assembly g_kl = C(N,l) * normalized g(k|l)  (Eq. 4, Eq. 2)
 *   - exact g_kl by brute-force enumeration (definition of g_kl, Eq. 2)
 *   - exact g_kl by a site-by-site transfer matrix, square lattice
 *   - thermodynamics from g_kl (Eq. 2 with the energy of Eq. 1)
 *
 * Fixed-point convention: ln g is kept as an int64 count of u = ln f_min,
 * ln f = F*u with F an integer; F starts at round(1/u) (f = e initially) and
 * each stage does F >>= 2 (ln f -> ln f / 4).  The walk stops when F == 0,
 * i.e. when ln f < ln f_min.
 *
 * Everything here is written for clarity, not speed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_SQUARE 0
#define OR_TRIANGULAR 1
#define OR_CUBIC 2
#define OR_SQUARE_OPEN 3      /* square lattice with open boundaries (Fig. 2) */

#define OR_MAXZ 6
#define OR_TABLE_N 4096

/* ------------------------------------------------------------------------ */
/* Lattices (Eq. 1: nearest-neighbour Ising model on an arbitrary lattice).  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int type, L, N, NB, z;
} or_lattice;

static int or_lat_make(or_lattice* lat, int type, int L)
{
    if (L < 3) return -1;            /* L >= 3: no double bonds on the torus */
    lat->type = type;
    lat->L = L;
    if (type == OR_SQUARE) {
        lat->N = L * L;
        lat->z = 4;
    } else if (type == OR_TRIANGULAR) {
        lat->N = L * L;
        lat->z = 6;
    } else if (type == OR_CUBIC) {
        lat->N = L * L * L;
        lat->z = 6;
    } else if (type == OR_SQUARE_OPEN) {
        lat->N = L * L;
        lat->z = 4;                          /* largest degree; edges have 3, corners 2 */
    } else {
        return -1;
    }
    lat->NB = type == OR_SQUARE_OPEN ? 2 * L * (L - 1) : lat->N * lat->z / 2;
    return 0;
}

/* Neighbours of site i.  Square: i = y*L + x, neighbours (x+-1, y), (x, y+-1).
 * Triangular (rhombic LxL torus): the square's four plus (x+1, y-1) and
 * (x-1, y+1).  Simple cubic: i = (zc*L + y)*L + x, +-1 along each axis.  All
 * periodic. */
static int or_neighbours(const or_lattice* lat, int i, int* nb)
{
    int L = lat->L;
    if (lat->type == OR_SQUARE_OPEN) {     /* no wrap: edge sites have fewer bonds */
        int x = i % L, y = i / L, d = 0;
        if (x + 1 < L) nb[d++] = i + 1;
        if (x > 0) nb[d++] = i - 1;
        if (y + 1 < L) nb[d++] = i + L;
        if (y > 0) nb[d++] = i - L;
        return d;
    }
    if (lat->type == OR_CUBIC) {
        int x = i % L, y = (i / L) % L, zc = i / (L * L);
        int xp = (x + 1) % L, xm = (x + L - 1) % L;
        int yp = (y + 1) % L, ym = (y + L - 1) % L;
        int zp = (zc + 1) % L, zm = (zc + L - 1) % L;
        nb[0] = (zc * L + y) * L + xp;
        nb[1] = (zc * L + y) * L + xm;
        nb[2] = (zc * L + yp) * L + x;
        nb[3] = (zc * L + ym) * L + x;
        nb[4] = (zp * L + y) * L + x;
        nb[5] = (zm * L + y) * L + x;
        return 6;
    }
    int x = i % L, y = i / L;
    int xp = (x + 1) % L, xm = (x + L - 1) % L;
    int yp = (y + 1) % L, ym = (y + L - 1) % L;
    nb[0] = y * L + xp;
    nb[1] = y * L + xm;
    nb[2] = yp * L + x;
    nb[3] = ym * L + x;
    if (lat->type == OR_TRIANGULAR) {
        nb[4] = ym * L + xp;
        nb[5] = yp * L + xm;
        return 6;
    }
    return 4;
}

int or_lattice_info(int type, int L, int* N, int* NB, int* z)
{
    or_lattice lat;
    if (or_lat_make(&lat, type, L)) return -1;
    *N = lat.N;
    *NB = lat.NB;
    *z = lat.z;
    return 0;
}

/* k of a full configuration: number of antiparallel ("unhappy") nearest-
 * neighbour pairs (the k of E_kl in Eq. 2).  Every bond is seen from both
 * ends, hence the division by two. */
static int64_t or_count_k(const or_lattice* lat, const uint8_t* s)
{
    int nb[OR_MAXZ];
    int64_t twice = 0;
    for (int i = 0; i < lat->N; i++) {
        int d = or_neighbours(lat, i, nb);
        for (int m = 0; m < d; m++) twice += (s[i] != s[nb[m]]);
    }
    return twice / 2;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition:   */
/* ten rounds; each round multiplies words 0 and 2 by fixed odd constants,   */
/* and the new state is (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped  */
/* by the Weyl constants between rounds.                                     */
/* ------------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform index in [0, n) from a 32-bit word: floor(r * n / 2^32). */
static uint32_t or_pick(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Exp threshold table for the fixed-point acceptance (Eq. 3).               */
/*                                                                          */
/* The acceptance probability of an uphill move is exp(-u*d), d the ln g    */
/* difference in units of u.  The table samples 2^32*exp(-x) at x_i =       */
/* (i*2^q)*u, i = 0..4095, q the smallest shift with 4095*2^q*u >= 32 ln 2, */
/* so the last entry is below one part in 2^32.  Entry values are the      */
/* exact value rounded half up, evaluated here in long double.              */
/* ------------------------------------------------------------------------ */

int or_exp_table_q(double u)
{
    long double need = 32.0L * logl(2.0L);
    for (int q = 0; q < 40; q++) {
        long double reach = 4095.0L * ldexpl(1.0L, q) * (long double)u;
        if (reach >= need) return q;
    }
    return -1;
}

int or_exp_table(double u, uint64_t* t, int* q_out)
{
    if (!(u >= 1e-10 && u <= 0.5)) return -1;
    int q = or_exp_table_q(u);
    if (q < 0) return -1;
    for (int i = 0; i < OR_TABLE_N; i++) {
        double x = (double)((uint64_t)i << q) * u;          /* one rounding */
        long double v = ldexpl(expl(-(long double)x), 32) + 0.5L;
        t[i] = (uint64_t)floorl(v);
    }
    *q_out = q;
    return 0;
}

/* Threshold T(d) for d > 0: linear interpolation between table entries. */
static uint64_t or_threshold(const uint64_t* t, int q, int64_t d)
{
    uint64_t i = (uint64_t)d >> q;
    if (i >= OR_TABLE_N - 1) return 0;
    uint64_t frac = (uint64_t)d & ((1ull << q) - 1ull);
    return t[i] - (((t[i] - t[i + 1]) * frac) >> q);
}

/* Exported for the tests: T(d) for a given u (0 when u is out of range). */
uint64_t or_threshold_of(double u, int64_t d)
{
    uint64_t t[OR_TABLE_N];
    int q;
    if (or_exp_table(u, t, &q) || d <= 0) return 0;
    return or_threshold(t, q, d);
}

/* ------------------------------------------------------------------------ */
/* One micromagnetic line: the Wang-Landau walk at fixed l.                  */
/* ------------------------------------------------------------------------ */

/* Spacing of the reachable k.  On the periodic lattices every site has even
 * degree, so k has the parity of z*l: k is always even and the bin of k is
 * k/2.  With open boundaries edge sites have odd degree and k takes every
 * value: the bin of k is k. */
static int or_kstep(int type) { return type == OR_SQUARE_OPEN ? 1 : 2; }

int or_lattice_kstep(int type) { return or_kstep(type); }

/* Bins hold k in [0, k_hi(l)] with the lattice's spacing, k_hi = min(z*min(l,
 * N-l), N_B): no more than z bonds per minority spin can be unhappy. */
int64_t or_line_nbins(int type, int L, int ell)
{
    or_lattice lat;
    if (or_lat_make(&lat, type, L)) return -1;
    if (ell < 0 || ell > lat.N) return -1;
    int lm = ell < lat.N - ell ? ell : lat.N - ell;
    int64_t khi = (int64_t)lat.z * lm;
    if (khi > lat.NB) khi = lat.NB;
    return khi / or_kstep(type) + 1;
}

/* Scalar state slots (int64), shared layout with the Python wrapper. */
enum {
    SC_K = 0,        /* current k                                         */
    SC_T,            /* move attempts made so far (the step counter)      */
    SC_F,            /* ln f in units of u                                */
    SC_STAGE,        /* number of completed flat histograms               */
    SC_ACCEPTS,      /* accepted proposals                                */
    SC_TSTAGE,       /* t at the start of the current stage               */
    SC_STATUS,       /* 0 running, 1 converged                            */
    SC_CHECKS,       /* flatness checks made                              */
    SC_COUNT
};

/* The initial state (text around Eq. 3): l up spins placed at random on an
 * otherwise down lattice, lists of up-spin and down-spin indices, g = 1
 * (ln g = 0) and h = 0.  The l up sites are the first l entries of a partial
 * Fisher-Yates shuffle of 0..N-1 driven by Philox counter (t, 0, 1, 0);
 * U = perm[0, l), D = perm[l, N) in the order the shuffle leaves them. */
static void or_line_init(const or_lattice* lat, int ell, uint32_t seed, double u,
                         int32_t* perm, uint8_t* spins, int64_t* sc,
                         int64_t* lng, int64_t* hist, uint8_t* visited, int64_t nbins)
{
    int N = lat->N;
    uint32_t key[2] = {(uint32_t)ell, seed};
    for (int i = 0; i < N; i++) perm[i] = i;
    for (int t = 0; t < ell && t < N - 1; t++) {
        uint32_t ctr[4] = {(uint32_t)t, 0u, 1u, 0u}, r[4];
        or_philox4x32_10(ctr, key, r);
        int j = t + (int)or_pick(r[0], (uint32_t)(N - t));
        int tmp = perm[t];
        perm[t] = perm[j];
        perm[j] = tmp;
    }
    for (int i = 0; i < N; i++) spins[i] = 0;
    for (int a = 0; a < ell; a++) spins[perm[a]] = 1;
    for (int64_t b = 0; b < nbins; b++) {
        lng[b] = 0;
        hist[b] = 0;
        visited[b] = 0;
    }
    for (int m = 0; m < SC_COUNT; m++) sc[m] = 0;
    sc[SC_K] = or_count_k(lat, spins);
    sc[SC_F] = llround(1.0 / u);          /* ln f = 1 initially (f = e) */
    if (ell == 0 || ell == N) {
        /* No exchange move exists: the line has the single state k = 0. */
        visited[sc[SC_K] / or_kstep(lat->type)] = 1;
        sc[SC_F] = 0;
        sc[SC_STATUS] = 1;
    }
}

/* Change of k when up-spin i and down-spin j are both flipped: recount every
 * bond that touches i or j before and after the flip. */
static int64_t or_delta_k(const or_lattice* lat, uint8_t* s, int i, int j)
{
    int nbi[OR_MAXZ], nbj[OR_MAXZ];
    int di = or_neighbours(lat, i, nbi);
    int dj = or_neighbours(lat, j, nbj);
    int64_t before = 0, after = 0;
    for (int m = 0; m < di; m++) before += (s[i] != s[nbi[m]]);
    for (int m = 0; m < dj; m++)
        if (nbj[m] != i) before += (s[j] != s[nbj[m]]);
    s[i] ^= 1;
    s[j] ^= 1;
    for (int m = 0; m < di; m++) after += (s[i] != s[nbi[m]]);
    for (int m = 0; m < dj; m++)
        if (nbj[m] != i) after += (s[j] != s[nbj[m]]);
    s[i] ^= 1;
    s[j] ^= 1;
    return after - before;
}

/* Flatness (the 80%/80% convention stated with the WL recap): at least a
 * fraction x of the visited bins hold at least x times the mean histogram
 * over visited bins.  x = flat_pm / 1000, evaluated exactly in integers:
 *   hist[b] >= x * S/n   <=>  1000 * n * hist[b] >= flat_pm * S
 *   c >= x * n           <=>  1000 * c >= flat_pm * n                     */
static int or_is_flat(const int64_t* hist, const uint8_t* visited, int64_t nbins, int flat_pm)
{
    int64_t n = 0, S = 0, c = 0;
    for (int64_t b = 0; b < nbins; b++)
        if (visited[b]) {
            n++;
            S += hist[b];
        }
    if (n == 0) return 0;
    /* products can pass 2^63 on long stages: compare in 128-bit integers */
    for (int64_t b = 0; b < nbins; b++)
        if (visited[b] && (__int128)1000 * n * hist[b] >= (__int128)flat_pm * S) c++;
    return 1000 * c >= (int64_t)flat_pm * n;
}

/* Exported for the tests: the flatness test on a given histogram. */
int or_flatness(const int64_t* hist, const uint8_t* visited, int64_t nbins, int flat_pm)
{
    return or_is_flat(hist, visited, nbins, flat_pm);
}

/* Run the walk on line ell until F == 0 (converged) or t == budget.
 *   mode 0: deterministic -- acceptance r2 < T(d) against the exp table
 *   mode 1: production   -- acceptance U53(r2, r3) < exp(-u d) in double
 * init != 0 prepares the initial state first; otherwise the state passed in
 * is continued.  Returns 0, or -1 on bad arguments. */
int or_line_run(int type, int L, int ell, uint32_t seed, double u, int64_t C, int flat_pm,
                int64_t budget, int mode, int init, int same_f_resets,
                int32_t* perm, uint8_t* spins, int64_t* sc,
                int64_t* lng, int64_t* hist, uint8_t* visited)
{
    or_lattice lat;
    if (or_lat_make(&lat, type, L)) return -1;
    if (ell < 0 || ell > lat.N / 2 || C < 1 || flat_pm < 1 || flat_pm > 1000) return -1;
    uint64_t table[OR_TABLE_N];
    int q;
    if (or_exp_table(u, table, &q)) return -1;
    int64_t nbins = or_line_nbins(type, L, ell);
    if (init) or_line_init(&lat, ell, seed, u, perm, spins, sc, lng, hist, visited, nbins);

    int N = lat.N;
    const int ks = or_kstep(type);
    int32_t* U = perm;          /* up-spin list   */
    int32_t* D = perm + ell;    /* down-spin list */
    uint32_t key[2] = {(uint32_t)ell, seed};

    while (sc[SC_STATUS] == 0 && sc[SC_T] < budget) {
        uint64_t t = (uint64_t)sc[SC_T];
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, 0u}, r[4];
        or_philox4x32_10(ctr, key, r);

        /* Propose: one random up spin and one random down spin, both flipped. */
        uint32_t a = or_pick(r[0], (uint32_t)ell);
        uint32_t b = or_pick(r[1], (uint32_t)(N - ell));
        int i = U[a], j = D[b];
        int64_t k = sc[SC_K];
        int64_t kp = k + or_delta_k(&lat, spins, i, j);

        /* Eq. 3: accept with probability min(g(k)/g(k'), 1). */
        int64_t d = lng[kp / ks] - lng[k / ks];
        int accept;
        if (d <= 0) {
            accept = 1;
        } else if (mode == 0) {
            accept = (uint64_t)r[2] < or_threshold(table, q, d);
        } else {
            double u53 = ((double)(r[2] >> 5) * 67108864.0 + (double)(r[3] >> 6)) / 9007199254740992.0;
            accept = u53 < exp(-u * (double)d);
        }
        if (accept) {
            U[a] = j;
            D[b] = i;
            spins[i] = 0;
            spins[j] = 1;
            sc[SC_K] = kp;
            sc[SC_ACCEPTS]++;
        }

        /* g(current) *= f, h(current) += 1 -- after an accept the current state
         * is the proposal, after a reject it is the old state. */
        int64_t bc = sc[SC_K] / ks;
        lng[bc] += sc[SC_F];
        hist[bc] += 1;
        visited[bc] = 1;
        sc[SC_T] = (int64_t)(t + 1);

        if (sc[SC_T] % C == 0) {
            sc[SC_CHECKS]++;
            int flat = or_is_flat(hist, visited, nbins, flat_pm);
            if (!flat && same_f_resets > 0 && (sc[SC_T] - sc[SC_TSTAGE]) / C <= same_f_resets) {
                /* The extra reset at unchanged f (the remark after Eq. 4 on
                 * spectrum ends): within the first same_f_resets checks of a
                 * stage a histogram that is not flat is reset and ln g
                 * normalised, f is kept. */
                int64_t mn = INT64_MAX;
                for (int64_t x = 0; x < nbins; x++)
                    if (visited[x] && lng[x] < mn) mn = lng[x];
                for (int64_t x = 0; x < nbins; x++) {
                    if (visited[x]) lng[x] -= mn;
                    hist[x] = 0;
                }
            }
            if (flat) {
                /* Histogram reset, normalization, f -> f^(1/4).  In fixed point
                 * the normalization of Eq. 4 is a constant shift of ln g; the
                 * exact integer shift that keeps the visited minimum at zero
                 * is used, and Eq. 4 itself is applied at assembly. */
                int64_t mn = INT64_MAX;
                for (int64_t x = 0; x < nbins; x++)
                    if (visited[x] && lng[x] < mn) mn = lng[x];
                for (int64_t x = 0; x < nbins; x++) {
                    if (visited[x]) lng[x] -= mn;
                    hist[x] = 0;
                }
                sc[SC_F] >>= 2;
                sc[SC_STAGE]++;
                sc[SC_TSTAGE] = sc[SC_T];
                if (sc[SC_F] == 0) sc[SC_STATUS] = 1;   /* ln f < ln f_min */
            }
        }
    }
    return 0;
}

/* Recount-based audit of a line state: k matches the spins, U holds exactly
 * the up spins and D the down spins, and together they are a permutation.
 * Returns 0 when consistent. */
int or_line_audit(int type, int L, int ell, const int32_t* perm, const uint8_t* spins, int64_t k)
{
    or_lattice lat;
    if (or_lat_make(&lat, type, L)) return -1;
    int N = lat.N;
    uint8_t* seen = calloc((size_t)N, 1);
    int bad = 0;
    for (int a = 0; a < N && !bad; a++) {
        int i = perm[a];
        if (i < 0 || i >= N || seen[i]) bad = 1;
        else {
            seen[i] = 1;
            if ((a < ell) != (spins[i] == 1)) bad = 2;
        }
    }
    free(seen);
    if (bad) return bad;
    uint8_t* s = malloc((size_t)N);
    memcpy(s, spins, (size_t)N);
    int64_t kk = or_count_k(&lat, s);
    free(s);
    return kk == k ? 0 : 3;
}

/* ------------------------------------------------------------------------ */
/* Assembly (Eq. 4 applied once, Eq. 2's g_kl): for the visited bins,       */
/*   ln g_kl = ln C(N,l) + u*lng[b] - ln sum_{visited j} exp(u*lng[j]),      */
/* summed in ascending bin order; unvisited bins get -infinity.             */
/* ------------------------------------------------------------------------ */

void or_assemble(int N, int ell, int64_t nbins, const int64_t* lng, const uint8_t* visited,
                 double u, double* out)
{
    double lnC = lgamma((double)N + 1.0) - lgamma((double)ell + 1.0) - lgamma((double)(N - ell) + 1.0);
    double mx = -INFINITY;
    for (int64_t b = 0; b < nbins; b++)
        if (visited[b] && u * (double)lng[b] > mx) mx = u * (double)lng[b];
    double s = 0.0;
    for (int64_t b = 0; b < nbins; b++)
        if (visited[b]) s += exp(u * (double)lng[b] - mx);
    double lse = mx + log(s);
    for (int64_t b = 0; b < nbins; b++)
        out[b] = visited[b] ? lnC + u * (double)lng[b] - lse : -INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Exact g_kl by enumerating every configuration (definition in Eq. 2).     */
/* g is (NB+1) x (N+1), row-major [k][l], counts stored as doubles.         */
/* ------------------------------------------------------------------------ */

int or_brute_force(int type, int L, double* g)
{
    or_lattice lat;
    if (or_lat_make(&lat, type, L)) return -1;
    int N = lat.N;
    if (N > 30) return -1;
    int nb[OR_MAXZ];
    int nbonds = 0;
    int* bi = malloc(sizeof(int) * (size_t)lat.NB);
    int* bj = malloc(sizeof(int) * (size_t)lat.NB);
    for (int i = 0; i < N; i++) {
        int d = or_neighbours(&lat, i, nb);
        for (int m = 0; m < d; m++)
            if (i < nb[m]) {
                bi[nbonds] = i;
                bj[nbonds] = nb[m];
                nbonds++;
            }
    }
    if (nbonds != lat.NB) {
        free(bi);
        free(bj);
        return -2;
    }
    memset(g, 0, sizeof(double) * (size_t)(lat.NB + 1) * (size_t)(N + 1));
    for (uint64_t cfg = 0; cfg < (1ull << N); cfg++) {
        int ell = __builtin_popcountll(cfg);
        int k = 0;
        for (int e = 0; e < nbonds; e++) k += (int)(((cfg >> bi[e]) ^ (cfg >> bj[e])) & 1ull);
        g[(size_t)k * (size_t)(N + 1) + (size_t)ell] += 1.0;
    }
    free(bi);
    free(bj);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact g_kl for the periodic LxL square lattice by a site-by-site         */
/* transfer matrix.  The first row sigma0 is fixed (its vertical wrap bonds */
/* close on it at the last row); the remaining sites are added in row-major */
/* order while the state is the last L spins added ("broken row").  Each    */
/* state carries a polynomial in (k, l); l is truncated at ell_max.  First  */
/* rows related by a horizontal translation or reflection give identical    */
/* contributions, so one representative per orbit is run, weighted by the  */
/* orbit size.  g is (NB+1) x (ell_max+1), row-major [k][l].                */
/* ------------------------------------------------------------------------ */

static uint32_t or_rowmap(uint32_t w, int L, int shift, int reflect)
{
    uint32_t out = 0;
    for (int x = 0; x < L; x++) {
        if (!((w >> x) & 1u)) continue;
        int xx = reflect ? (L - 1 - x) : x;
        xx = (xx + shift) % L;
        out |= 1u << xx;
    }
    return out;
}

static void or_tm_one_row0(int L, int ell_max, uint32_t row0, double mult, double* gacc)
{
    int S = 1 << L;
    int NB = 2 * L * L;
    int KW = NB + 1, LW = ell_max + 1;
    size_t P = (size_t)KW * (size_t)LW;
    int l0 = __builtin_popcount(row0);
    if (l0 > ell_max) return;
    double* V = calloc((size_t)S * P, sizeof(double));
    double* t0 = calloc(P, sizeof(double));
    double* t1 = calloc(P, sizeof(double));
    int k0 = 0;
    for (int x = 0; x < L; x++) k0 += (int)(((row0 >> x) ^ (row0 >> ((x + 1) % L))) & 1u);
    V[(size_t)row0 * P + (size_t)k0 * LW + (size_t)l0] = 1.0;
    int kmax = k0, lmax = l0;
    for (int y = 1; y < L; y++) {
        for (int x = 0; x < L; x++) {
            uint32_t bit = 1u << x;
            int kadd = 1 + (x >= 1) + (x == L - 1) + (y == L - 1);
            int kmax_new = kmax + kadd > NB ? NB : kmax + kadd;
            int lmax_new = lmax + 1 > ell_max ? ell_max : lmax + 1;
            /* live box after this site: k in [0, kmax_new], l in [0, lmax_new] */
            size_t live = (size_t)(kmax_new + 1) * LW;
            for (uint32_t w = 0; w < (uint32_t)S; w++) {
                if (w & bit) continue;
                double* A = V + (size_t)w * P;            /* old spin (x, y-1) = 0 */
                double* B = V + (size_t)(w | bit) * P;    /* old spin (x, y-1) = 1 */
                memset(t0, 0, live * sizeof(double));
                memset(t1, 0, live * sizeof(double));
                for (int s = 0; s <= 1; s++) {
                    /* bonds closed by the new spin s at (x, y): up, left,
                     * right-wrap (x = L-1 meets (0, y)), down-wrap (last row
                     * meets the first row) */
                    int others = 0;
                    if (x >= 1) others += (s != (int)((w >> (x - 1)) & 1u));
                    if (x == L - 1) others += (s != (int)(w & 1u));
                    if (y == L - 1) others += (s != (int)((row0 >> x) & 1u));
                    int dkA = others + (s != 0);
                    int dkB = others + (s != 1);
                    double* T = s ? t1 : t0;
                    int ltop = lmax + s > ell_max ? ell_max - s : lmax;
                    for (int k = 0; k <= kmax; k++) {
                        const double* a = A + (size_t)k * LW;
                        const double* b = B + (size_t)k * LW;
                        double* ta = T + (size_t)(k + dkA) * LW + s;
                        double* tb = T + (size_t)(k + dkB) * LW + s;
                        for (int l = 0; l <= ltop; l++) ta[l] += a[l];
                        for (int l = 0; l <= ltop; l++) tb[l] += b[l];
                    }
                }
                memcpy(A, t0, live * sizeof(double));
                memcpy(B, t1, live * sizeof(double));
            }
            kmax = kmax_new;
            lmax = lmax_new;
        }
    }
    for (uint32_t w = 0; w < (uint32_t)S; w++) {
        double* A = V + (size_t)w * P;
        for (size_t p = 0; p < P; p++) gacc[p] += mult * A[p];
    }
    free(V);
    free(t0);
    free(t1);
}

int or_tm_square(int L, int ell_max, double* g, int nthreads)
{
    if (L < 3 || L > 14) return -1;
    int N = L * L, NB = 2 * L * L;
    if (ell_max < 0 || ell_max > N) return -1;
    size_t P = (size_t)(NB + 1) * (size_t)(ell_max + 1);
    memset(g, 0, P * sizeof(double));
    int S = 1 << L;
    /* representatives: the smallest member of each translation/reflection orbit */
    uint32_t* rep = malloc(sizeof(uint32_t) * (size_t)S);
    double* mult = malloc(sizeof(double) * (size_t)S);
    int nrep = 0;
    for (uint32_t w = 0; w < (uint32_t)S; w++) {
        int is_min = 1;
        uint32_t orbit[64];
        int norbit = 0;
        for (int refl = 0; refl <= 1; refl++)
            for (int sh = 0; sh < L; sh++) {
                uint32_t v = or_rowmap(w, L, sh, refl);
                if (v < w) is_min = 0;
                int dup = 0;
                for (int o = 0; o < norbit; o++)
                    if (orbit[o] == v) dup = 1;
                if (!dup) orbit[norbit++] = v;
            }
        if (is_min) {
            rep[nrep] = w;
            mult[nrep] = (double)norbit;
            nrep++;
        }
    }
    if (nthreads < 1) nthreads = 1;
    double* part = calloc((size_t)nthreads * P, sizeof(double));
    /* Fixed assignment of representatives to partial sums, so the result
     * does not depend on thread timing. */
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
    for (int th = 0; th < nthreads; th++)
        for (int r = th; r < nrep; r += nthreads)
            or_tm_one_row0(L, ell_max, rep[r], mult[r], part + (size_t)th * P);
    for (int th = 0; th < nthreads; th++)
        for (size_t p = 0; p < P; p++) g[p] += part[(size_t)th * P + p];
    free(part);
    free(rep);
    free(mult);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Thermodynamics from the density of states (Eq. 2): for each temperature  */
/* T (J = 1, k_B = 1) and field H,                                           */
/*   Z = sum_{k,l} g_kl exp(-E_kl / T),  E_kl = -(N_B - 2k) - H M,           */
/* M = sum_i S_i = 2l - N for l up spins (Eq. 1; the field term printed with */
/* Eq. 2 has the opposite sign, which only mirrors <M>).  Input: ln g over   */
/* lines l = 0..N/2 (ragged, offsets of                                      */
/* length N/2 + 2, bin b holding k = b*kstep, -inf where g = 0); line        */
/* l > N/2 is line N - l.  Output per (T, H), row-major [iT][iH][6]:          */
/*   ln Z / N, <E>/N, C/N = (<E^2> - <E>^2)/(N T^2), <M>/N, <|M|>/N,          */
/*   chi/N = (<M^2> - <M>^2)/(N T).                                           */
/* ------------------------------------------------------------------------ */

void or_thermo(int N, int NB, const int64_t* offsets, const double* lng, int kstep,
               const double* T, int nT, const double* H, int nH, double* out)
{
    int half = N / 2;
    for (int a = 0; a < nT; a++)
        for (int c = 0; c < nH; c++) {
            double beta = 1.0 / T[a], h = H[c];
            double mx = -INFINITY;
            for (int l = 0; l <= N; l++) {
                int src = l <= half ? l : N - l;
                for (int64_t b = offsets[src]; b < offsets[src + 1]; b++) {
                    if (isinf(lng[b])) continue;
                    int64_t k = (b - offsets[src]) * kstep;
                    double E = -(double)(NB - 2 * k) - h * (double)(2 * l - N);
                    double x = lng[b] - beta * E;
                    if (x > mx) mx = x;
                }
            }
            double z = 0, e1 = 0, e2 = 0, m1 = 0, ma = 0, m2 = 0;
            for (int l = 0; l <= N; l++) {
                int src = l <= half ? l : N - l;
                for (int64_t b = offsets[src]; b < offsets[src + 1]; b++) {
                    if (isinf(lng[b])) continue;
                    int64_t k = (b - offsets[src]) * kstep;
                    double M = (double)(2 * l - N);
                    double E = -(double)(NB - 2 * k) - h * M;
                    double w = exp(lng[b] - beta * E - mx);
                    z += w;
                    e1 += w * E;
                    e2 += w * E * E;
                    m1 += w * M;
                    ma += w * fabs(M);
                    m2 += w * M * M;
                }
            }
            e1 /= z; e2 /= z; m1 /= z; ma /= z; m2 /= z;
            double* o = out + ((size_t)a * nH + c) * 6;
            o[0] = (mx + log(z)) / N;
            o[1] = e1 / N;
            o[2] = (e2 - e1 * e1) * beta * beta / N;
            o[3] = m1 / N;
            o[4] = ma / N;
            o[5] = (m2 - m1 * m1) * beta / N;
        }
}
