/*
 * Reference oracle for the bmDCA hot path (adabmDCA 2.0, arXiv 2501.18456).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
 * FP64 restatement of the paper's equations.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  The CUDA
 * library shares no code, header, table or helper with it.
 *
 * Conventions (readings of the paper where it is silent are listed in the
 * design notes; each is repeated next to the function it affects):
 *   - a sequence / chain state is s[0..L-1], s_i in {0..q-1}, gap = 0
 *     (Sec. 2.3, Table 1: the gap is the first symbol of every alphabet);
 *   - couplings use the natural layout J[i][j][a][b] = J_ij(a,b), FP64,
 *     symmetric J_ij(a,b) = J_ji(b,a), J_ii = 0 (Sec. 2.1, after Eq. 1);
 *   - fields h[i][a] = h_i(a);
 *   - energy E(s) = -sum_i h_i(s_i) - sum_{i<j} J_ij(s_i,s_j), so that
 *     p(s) ~ exp(-E(s)) (Eq. 1); each unordered pair counted once;
 *   - chains are unweighted model samples (Sec. 2.1, "Monte Carlo
 *     estimation of the gradient").
 *
 * Every function is pinned by the CPU tests against something other than
 * itself (exact enumeration, closed forms, numpy brute force, numpy's
 * independent Philox implementation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------
 * Philox4x64-10 counter-based generator, from its published definition
 * (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2,
 * 3", SC'11).  Ten rounds; each round multiplies counter words 0 and 2 by
 * the two Philox multipliers, takes the high/low halves of the 128-bit
 * products and mixes them with the other counter words and the round key.
 * The key is bumped by the two Weyl constants between rounds.
 * The paper itself only says chains are updated with Gibbs steps; the
 * generator is this library's choice so that both sides can draw the same
 * uniforms (keyed by seed, chain, sweep and site).
 * ---------------------------------------------------------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        uint64_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* The 24-bit uniform used by every draw: key = (seed, 0), counter =
 * (chain, sweep, site, tag); the top 24 bits of output word 0.
 * tag 0 = Gibbs draw, tag 1 = chain initialisation. */
uint32_t orc_u24(uint64_t seed, uint64_t chain, uint64_t sweep, uint64_t site, uint64_t tag)
{
    uint64_t ctr[4] = {chain, sweep, site, tag};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    return (uint32_t)(out[0] >> 40);
}

/* ------------------------------------------------------------------------
 * Chain initialisation: uniformly random sequences (Sec. 2.1, chains
 * "chosen uniformly at random").  Symbol = floor(u24 * q / 2^24), exact in
 * integer arithmetic.  chain0 offsets the chain index so that a subset of
 * chains can be generated.
 * ---------------------------------------------------------------------- */
void orc_chains_init(int M, int L, int q, uint64_t seed, uint64_t chain0, uint8_t *s)
{
    for (int m = 0; m < M; ++m)
        for (int i = 0; i < L; ++i) {
            uint64_t r = orc_u24(seed, chain0 + (uint64_t)m, 0, (uint64_t)i, 1);
            s[(size_t)m * L + i] = (uint8_t)((r * (uint64_t)q) >> 24);
        }
}

static inline size_t jidx(int L, int q, int i, int j, int a, int b)
{
    return (((size_t)i * L + j) * q + a) * q + b;
}

/* ------------------------------------------------------------------------
 * DCA energy, Eq. 1: E(s) = -sum_i h_i(s_i) - sum_{i<j} J_ij(s_i, s_j).
 * ---------------------------------------------------------------------- */
double orc_energy(const double *h, const double *J, int L, int q, const uint8_t *s)
{
    double e = 0.0;
    for (int i = 0; i < L; ++i) e -= h[(size_t)i * q + s[i]];
    for (int i = 0; i < L; ++i)
        for (int j = i + 1; j < L; ++j) e -= J[jidx(L, q, i, j, s[i], s[j])];
    return e;
}

void orc_energy_batch(const double *h, const double *J, int L, int q, const uint8_t *S, int n, double *E)
{
    for (int k = 0; k < n; ++k) E[k] = orc_energy(h, J, L, q, S + (size_t)k * L);
}

/* Local field of site i given the rest of the sequence (the conditional of
 * Eq. 1 with every other site fixed):
 * H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j), summed over j ascending. */
void orc_fields(const double *h, const double *J, int L, int q, const uint8_t *s, int i, double *H)
{
    for (int a = 0; a < q; ++a) {
        double acc = h[(size_t)i * q + a];
        for (int j = 0; j < L; ++j) {
            if (j == i) continue;
            acc += J[jidx(L, q, i, j, a, s[j])];
        }
        H[a] = acc;
    }
}

/* Categorical draw by inverse CDF from p(a) ~ exp(beta * H(a)) with the
 * uniform u in [0,1).  Reading (the paper gives no draw rule): subtract the
 * maximum for range safety, prefix-sum the weights for a ascending, pick
 * the first a with u * S_total < S_a (q-1 if none).  *margin receives the
 * distance of u to the nearest interior CDF boundary S_a / S_total. */
int orc_draw(const double *H, int q, double beta, double u, double *margin)
{
    double w[64], S[64];
    double mx = -INFINITY;
    for (int a = 0; a < q; ++a) if (beta * H[a] > mx) mx = beta * H[a];
    double acc = 0.0;
    for (int a = 0; a < q; ++a) {
        w[a] = exp(beta * H[a] - mx);
        acc += w[a];
        S[a] = acc;
    }
    double t = u * S[q - 1];
    int pick = q - 1;
    for (int a = 0; a < q; ++a)
        if (t < S[a]) { pick = a; break; }
    if (margin) {
        double mg = INFINITY;
        for (int a = 0; a < q - 1; ++a) {
            double d = fabs(u - S[a] / S[q - 1]);
            if (d < mg) mg = d;
        }
        *margin = mg;
    }
    return pick;
}

/* Conditional distribution P(s_i = a | s_{-i}) at inverse temperature beta. */
void orc_conditional(const double *h, const double *J, int L, int q, const uint8_t *s, int i,
                     double beta, double *P)
{
    double H[64];
    orc_fields(h, J, L, q, s, i, H);
    double mx = -INFINITY, Z = 0.0;
    for (int a = 0; a < q; ++a) if (beta * H[a] > mx) mx = beta * H[a];
    for (int a = 0; a < q; ++a) { P[a] = exp(beta * H[a] - mx); Z += P[a]; }
    for (int a = 0; a < q; ++a) P[a] /= Z;
}

/* ------------------------------------------------------------------------
 * Persistent-chain Gibbs sampling (Sec. 2.1, "Monte Carlo estimation of
 * the gradient"; a sweep proposes every site once, Sec. 3.3 "Number of
 * Monte Carlo steps").  Reading: sites visited in order 0..L-1 every sweep;
 * sweep counter = sweep0 + k, never repeated over a run.
 * ---------------------------------------------------------------------- */
void orc_gibbs(const double *h, const double *J, int L, int q, int M, uint8_t *S,
               uint64_t seed, uint64_t chain0, uint64_t sweep0, int nsweeps, double beta)
{
    double H[64];
    for (int k = 0; k < nsweeps; ++k)
        for (int m = 0; m < M; ++m) {
            uint8_t *s = S + (size_t)m * L;
            for (int i = 0; i < L; ++i) {
                orc_fields(h, J, L, q, s, i, H);
                uint32_t r = orc_u24(seed, chain0 + (uint64_t)m, sweep0 + (uint64_t)k, (uint64_t)i, 0);
                double u = (double)r * (1.0 / 16777216.0);
                s[i] = (uint8_t)orc_draw(H, q, beta, u, NULL);
            }
        }
}

/* Teacher-forced check of one sweep produced elsewhere.  For every chain
 * and site i (in order) the oracle conditions on after[j] for j < i and on
 * before[j] for j > i -- exactly what a correct sequential sweep conditions
 * on -- draws with the same uniform and compares with after[i].
 * Returns the number of site-updates that disagree; *max_margin receives
 * the largest oracle margin among the disagreements (0 if none) and
 * *min_margin the smallest margin over all site-updates.  The first `cap`
 * disagreements are recorded (chain index relative to `before`, site,
 * oracle margin, symbol found, symbol the oracle draws) when the record
 * arrays are given, so that every boundary flip can be reported. */
long orc_gibbs_verify_rec(const double *h, const double *J, int L, int q, int M,
                          const uint8_t *before, const uint8_t *after, uint64_t seed,
                          uint64_t chain0, uint64_t sweep, double beta,
                          double *max_margin, double *min_margin, long cap,
                          int64_t *rec_chain, int32_t *rec_site, double *rec_margin,
                          int32_t *rec_got, int32_t *rec_want)
{
    double H[64];
    uint8_t *s = (uint8_t *)malloc((size_t)L);
    long bad = 0;
    double mxm = 0.0, mnm = INFINITY;
    for (int m = 0; m < M; ++m) {
        memcpy(s, before + (size_t)m * L, (size_t)L);
        for (int i = 0; i < L; ++i) {
            orc_fields(h, J, L, q, s, i, H);
            uint32_t r = orc_u24(seed, chain0 + (uint64_t)m, sweep, (uint64_t)i, 0);
            double u = (double)r * (1.0 / 16777216.0);
            double mg;
            int pick = orc_draw(H, q, beta, u, &mg);
            if (mg < mnm) mnm = mg;
            uint8_t got = after[(size_t)m * L + i];
            if (got != pick) {
                if (bad < cap && rec_chain) {
                    rec_chain[bad] = m;
                    rec_site[bad] = i;
                    rec_margin[bad] = mg;
                    rec_got[bad] = got;
                    rec_want[bad] = pick;
                }
                ++bad;
                if (mg > mxm) mxm = mg;
            }
            s[i] = got;
        }
    }
    free(s);
    if (max_margin) *max_margin = mxm;
    if (min_margin) *min_margin = mnm;
    return bad;
}

long orc_gibbs_verify(const double *h, const double *J, int L, int q, int M,
                      const uint8_t *before, const uint8_t *after, uint64_t seed,
                      uint64_t chain0, uint64_t sweep, double beta,
                      double *max_margin, double *min_margin)
{
    return orc_gibbs_verify_rec(h, J, L, q, M, before, after, seed, chain0, sweep, beta,
                                max_margin, min_margin, 0, NULL, NULL, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------
 * Metropolis-Hastings sweeps (Sec. 2.1: chains are updated "using Gibbs or
 * Metropolis-Hastings sampling steps"; the --sampler option of the
 * training and sampling commands).  The paper states no proposal; the
 * readings taken here:
 *   - sites visited in order 0..L-1, one proposal per site per sweep;
 *   - proposal a' uniform over the q-1 symbols other than the current s_i
 *     (symmetric, so the Hastings ratio is the Boltzmann ratio):
 *     k = floor(u24_p (q-1) / 2^24) from Philox tag 2, a' = k + (k >= s_i);
 *   - acceptance with probability min(1, exp(beta (H_i(a') - H_i(s_i)))),
 *     H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j): accepted iff
 *     u_a < exp(beta dH), u_a = u24_a / 2^24 from Philox tag 3 (dH >= 0 is
 *     always accepted since u_a < 1);
 *   - q = 1: nothing to propose, the state is kept.
 * The margin of a decision is |u_a - min(1, exp(beta dH))|.
 * ---------------------------------------------------------------------- */
static int orc_metropolis_step(const double *h, const double *J, int L, int q, const uint8_t *s, int i,
                               double beta, uint64_t seed, uint64_t chain, uint64_t sweep, double *margin)
{
    if (q < 2) {
        if (margin) *margin = INFINITY;
        return s[i];
    }
    double H[64];
    orc_fields(h, J, L, q, s, i, H);
    const uint32_t rp = orc_u24(seed, chain, sweep, (uint64_t)i, 2);
    const uint32_t ra = orc_u24(seed, chain, sweep, (uint64_t)i, 3);
    int prop = (int)(((uint64_t)rp * (uint64_t)(q - 1)) >> 24);
    if (prop >= s[i]) prop += 1;
    const double dH = H[prop] - H[s[i]];
    const double pacc = dH >= 0.0 ? 1.0 : exp(beta * dH);
    const double u = (double)ra * (1.0 / 16777216.0);
    if (margin) *margin = fabs(u - pacc);
    return u < pacc ? prop : s[i];
}

void orc_metropolis(const double *h, const double *J, int L, int q, int M, uint8_t *S, uint64_t seed,
                    uint64_t chain0, uint64_t sweep0, int nsweeps, double beta)
{
    for (int k = 0; k < nsweeps; ++k)
        for (int m = 0; m < M; ++m) {
            uint8_t *s = S + (size_t)m * L;
            for (int i = 0; i < L; ++i)
                s[i] = (uint8_t)orc_metropolis_step(h, J, L, q, s, i, beta, seed, chain0 + (uint64_t)m,
                                                    sweep0 + (uint64_t)k, NULL);
        }
}

/* Teacher-forced check of one Metropolis sweep produced elsewhere, as
 * orc_gibbs_verify_rec: the oracle conditions on after[j] for j < i and
 * before[j] for j > i, proposes and decides with the same uniforms and
 * compares with after[i]; disagreements are counted and recorded. */
long orc_metropolis_verify_rec(const double *h, const double *J, int L, int q, int M, const uint8_t *before,
                               const uint8_t *after, uint64_t seed, uint64_t chain0, uint64_t sweep, double beta,
                               double *max_margin, double *min_margin, long cap, int64_t *rec_chain,
                               int32_t *rec_site, double *rec_margin, int32_t *rec_got, int32_t *rec_want)
{
    uint8_t *s = (uint8_t *)malloc((size_t)L);
    long bad = 0;
    double mxm = 0.0, mnm = INFINITY;
    for (int m = 0; m < M; ++m) {
        memcpy(s, before + (size_t)m * L, (size_t)L);
        for (int i = 0; i < L; ++i) {
            double mg;
            const int want = orc_metropolis_step(h, J, L, q, s, i, beta, seed, chain0 + (uint64_t)m, sweep, &mg);
            if (mg < mnm) mnm = mg;
            const uint8_t got = after[(size_t)m * L + i];
            if (got != want) {
                if (bad < cap && rec_chain) {
                    rec_chain[bad] = m;
                    rec_site[bad] = i;
                    rec_margin[bad] = mg;
                    rec_got[bad] = got;
                    rec_want[bad] = want;
                }
                ++bad;
                if (mg > mxm) mxm = mg;
            }
            s[i] = got;
        }
    }
    free(s);
    if (max_margin) *max_margin = mxm;
    if (min_margin) *min_margin = mnm;
    return bad;
}

/* ------------------------------------------------------------------------
 * Model statistics from the chains, unweighted (Sec. 2.1: p_i, p_ij are
 * estimated by the chain frequencies).  Integer counts over the upper
 * block triangle i <= j, block (i,j) at index i*L - i*(i-1)/2 + (j-i),
 * each block q x q row-major [a][b] = #{m : s_i = a, s_j = b}.
 * ---------------------------------------------------------------------- */
void orc_chain_stats(const uint8_t *S, int M, int L, int q, int32_t *C)
{
    size_t nblk = (size_t)L * (L + 1) / 2;
    memset(C, 0, nblk * q * q * sizeof(int32_t));
    for (int m = 0; m < M; ++m) {
        const uint8_t *s = S + (size_t)m * L;
        for (int i = 0; i < L; ++i)
            for (int j = i; j < L; ++j) {
                size_t p = (size_t)i * L - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
                C[p * q * q + (size_t)s[i] * q + s[j]] += 1;
            }
    }
}

/* ------------------------------------------------------------------------
 * Importance weights, Eq. 7 (Sec. 2.3): w_m = 1 / N_m with N_m the number
 * of sequences n (m itself included) whose identity with m -- the count of
 * positions with equal symbols, gaps included -- is at least thr.
 * The caller passes the integer threshold thr = ceil(seqid * L).
 * M_eff = sum_m w_m (Sec. 3.3, "Regularization").
 * ---------------------------------------------------------------------- */
void orc_seq_weights(const uint8_t *X, int N, int L, int thr, double *w, double *meff)
{
    double tot = 0.0;
    for (int m = 0; m < N; ++m) {
        long cnt = 0;
        for (int n = 0; n < N; ++n) {
            int id = 0;
            for (int i = 0; i < L; ++i) id += (X[(size_t)m * L + i] == X[(size_t)n * L + i]);
            if (id >= thr) ++cnt;
        }
        w[m] = 1.0 / (double)cnt;
    }
    for (int m = 0; m < N; ++m) tot += w[m];
    *meff = tot;
}

/* ------------------------------------------------------------------------
 * Weighted data frequencies, Eq. 3, followed by the pseudocount of
 * Eqs. 8-9: f_i = (1-alpha) f_i^data + alpha/q,
 *            f_ij = (1-alpha) f_ij^data + alpha/q^2  (i != j).
 * w == NULL means uniform weights (M_eff = N).  Full layout
 * fij[i][j][a][b]; reading for the unused diagonal blocks:
 * fij[i][i][a][b] = delta_ab f_i(a).
 * ---------------------------------------------------------------------- */
void orc_data_stats(const uint8_t *X, const double *w, int N, int L, int q, double alpha,
                    double *fi, double *fij)
{
    double meff = 0.0;
    for (int m = 0; m < N; ++m) meff += w ? w[m] : 1.0;
    memset(fi, 0, (size_t)L * q * sizeof(double));
    memset(fij, 0, (size_t)L * L * q * q * sizeof(double));
    for (int m = 0; m < N; ++m) {
        double wm = w ? w[m] : 1.0;
        const uint8_t *s = X + (size_t)m * L;
        for (int i = 0; i < L; ++i) {
            fi[(size_t)i * q + s[i]] += wm;
            for (int j = 0; j < L; ++j)
                if (j != i) fij[jidx(L, q, i, j, s[i], s[j])] += wm;
        }
    }
    for (size_t k = 0; k < (size_t)L * q; ++k) fi[k] = (1.0 - alpha) * (fi[k] / meff) + alpha / q;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j)
            for (int a = 0; a < q; ++a)
                for (int b = 0; b < q; ++b) {
                    size_t k = jidx(L, q, i, j, a, b);
                    if (i == j)
                        fij[k] = (a == b) ? fi[(size_t)i * q + a] : 0.0;
                    else
                        fij[k] = (1.0 - alpha) * (fij[k] / meff) + alpha / ((double)q * q);
                }
}

/* ------------------------------------------------------------------------
 * Convergence check (Sec. 2.1, "Convergence criterium"): Pearson
 * correlation between C^data_ij(a,b) = f_ij(a,b) - f_i(a) f_j(b) and
 * C^model_ij(a,b) = p_ij(a,b) - p_i(a) p_j(b), over i < j and all (a,b).
 * p from the chain counts C (layout of orc_chain_stats) divided by M.
 * Plain two-pass formula (means first, then centred sums).
 * ---------------------------------------------------------------------- */
static double *orc_single_from_counts(const int32_t *C, int M, int L, int q)
{
    double *pi = (double *)malloc((size_t)L * q * sizeof(double));
    for (int i = 0; i < L; ++i) {
        size_t p = (size_t)i * L - (size_t)i * (i - 1) / 2;   /* diagonal block (i,i) */
        for (int a = 0; a < q; ++a) {
            long c = 0;
            for (int b = 0; b < q; ++b) c += C[p * q * q + (size_t)a * q + b];
            pi[(size_t)i * q + a] = (double)c / M;
        }
    }
    return pi;
}

double orc_pearson(const double *fi, const double *fij, const int32_t *C, int M, int L, int q)
{
    double *pi = orc_single_from_counts(C, M, L, q);
    double n = 0.0, sx = 0.0, sy = 0.0;
    /* pass 1: means */
    for (int i = 0; i < L; ++i)
        for (int j = i + 1; j < L; ++j) {
            size_t p = (size_t)i * L - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
            for (int a = 0; a < q; ++a)
                for (int b = 0; b < q; ++b) {
                    double x = fij[jidx(L, q, i, j, a, b)] - fi[(size_t)i * q + a] * fi[(size_t)j * q + b];
                    double y = (double)C[p * q * q + (size_t)a * q + b] / M
                               - pi[(size_t)i * q + a] * pi[(size_t)j * q + b];
                    sx += x; sy += y; n += 1.0;
                }
        }
    double mx = sx / n, my = sy / n;
    double sxx = 0.0, syy = 0.0, sxy = 0.0;
    /* pass 2: centred second moments */
    for (int i = 0; i < L; ++i)
        for (int j = i + 1; j < L; ++j) {
            size_t p = (size_t)i * L - (size_t)i * (i - 1) / 2 + (size_t)(j - i);
            for (int a = 0; a < q; ++a)
                for (int b = 0; b < q; ++b) {
                    double x = fij[jidx(L, q, i, j, a, b)] - fi[(size_t)i * q + a] * fi[(size_t)j * q + b];
                    double y = (double)C[p * q * q + (size_t)a * q + b] / M
                               - pi[(size_t)i * q + a] * pi[(size_t)j * q + b];
                    sxx += (x - mx) * (x - mx);
                    syy += (y - my) * (y - my);
                    sxy += (x - mx) * (y - my);
                }
        }
    free(pi);
    return sxy / sqrt(sxx * syy);
}

/* ------------------------------------------------------------------------
 * Boltzmann-learning step, Eq. 5 ("params update"):
 *   h_i(a)    += lr (f_i(a)    - p_i(a))
 *   J_ij(a,b) += lr (f_ij(a,b) - p_ij(a,b))   for i != j; J_ii stays 0.
 * p from the counts (layout of orc_chain_stats) divided by M; the (j,i)
 * entry is the same pair statistic transposed, keeping J symmetric.
 * ---------------------------------------------------------------------- */
void orc_update(double *h, double *J, const double *fi, const double *fij, const int32_t *C,
                int M, double lr, int L, int q)
{
    double *pi = orc_single_from_counts(C, M, L, q);
    for (size_t k = 0; k < (size_t)L * q; ++k) h[k] += lr * (fi[k] - pi[k]);
    free(pi);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            if (i == j) continue;
            int lo = i < j ? i : j, hi = i < j ? j : i;
            size_t p = (size_t)lo * L - (size_t)lo * (lo - 1) / 2 + (size_t)(hi - lo);
            for (int a = 0; a < q; ++a)
                for (int b = 0; b < q; ++b) {
                    int32_t c = (i < j) ? C[p * q * q + (size_t)a * q + b] : C[p * q * q + (size_t)b * q + a];
                    J[jidx(L, q, i, j, a, b)] += lr * (fij[jidx(L, q, i, j, a, b)] - (double)c / M);
                }
        }
}

/* ------------------------------------------------------------------------
 * Single-mutant library (Sec. 4.4): dE(i,a) = E(wt with s_i = a) - E(wt),
 * computed by evaluating both energies by definition.  dE(i, wt_i) = 0.
 * Output layout dE[i][a].
 * ---------------------------------------------------------------------- */
void orc_mutant_scan(const double *h, const double *J, int L, int q, const uint8_t *wt, double *dE)
{
    uint8_t *s = (uint8_t *)malloc((size_t)L);
    double e0 = orc_energy(h, J, L, q, wt);
    for (int i = 0; i < L; ++i)
        for (int a = 0; a < q; ++a) {
            memcpy(s, wt, (size_t)L);
            s[i] = (uint8_t)a;
            dE[(size_t)i * q + a] = (a == wt[i]) ? 0.0 : orc_energy(h, J, L, q, s) - e0;
        }
    free(s);
}

/* ------------------------------------------------------------------------
 * Sparse interaction graphs (Sec. 2.2, "Training sparse models").
 *
 * An element is one coupling entry J_ij(a,b) with i < j; its mirror
 * J_ji(b,a) follows it.  Elements are numbered in row order: pairs (i,j),
 * i < j, in the order (0,1), (0,2), ..., (1,2), ..., and within a pair a*q+b.
 * `active` uses the natural layout [i][j][a][b] and is kept symmetric.
 * ---------------------------------------------------------------------- */
static size_t orc_n_elements(int L, int q) { return (size_t)L * (L - 1) / 2 * q * q; }

/* (i, j, a, b) of element e. */
static void orc_element(size_t e, int L, int q, int *i, int *j, int *a, int *b)
{
    const size_t qq = (size_t)q * q;
    size_t p = e / qq, w = e % qq;
    int r = 0;
    while (p >= (size_t)(L - 1 - r)) {
        p -= (size_t)(L - 1 - r);
        ++r;
    }
    *i = r;
    *j = r + 1 + (int)p;
    *a = (int)(w / q);
    *b = (int)(w % q);
}

/* Element decimation (edDCA): the score of removing an active element is
 * the symmetric Kullback-Leibler divergence between the model P and the
 * model P' with that element set to zero.  Removing it multiplies P(s) by
 * e^{-J} where s_i = a and s_j = b (then renormalises), so with p = p_ij(a,b)
 * of the model
 *   p' = p e^{-J} / (1 - p + p e^{-J}),
 *   KL(P||P') + KL(P'||P) = J (p - p').
 * Reading: the paper names this criterion and leaves its evaluation to the
 * literature; this is its exact value for one element given p.  Negative
 * values from rounding are taken as 0.  Inactive elements score +inf.
 * pij: model pair frequencies, natural layout [i][j][a][b]. */
void orc_decimation_scores(const double *J, const double *pij, const uint8_t *active, int L, int q,
                           double *score)
{
    const size_t n = orc_n_elements(L, q);
    for (size_t e = 0; e < n; ++e) {
        int i, j, a, b;
        orc_element(e, L, q, &i, &j, &a, &b);
        const size_t x = jidx(L, q, i, j, a, b);
        if (!active[x]) {
            score[e] = INFINITY;
            continue;
        }
        const double Jx = J[x], p = pij[x];
        const double w = p * exp(-Jx);
        const double pp = w / (1.0 - p + w);
        const double d = Jx * (p - pp);
        score[e] = d > 0.0 ? d : 0.0;
    }
}

/* Element activation (eaDCA): the score of an element is how far the
 * model's pair frequency p = p_ij(a,b) is from the data's f = f_ij(a,b),
 * measured by the Bernoulli Kullback-Leibler divergence
 *   A = f log(f/p) + (1-f) log((1-f)/(1-p)),   0 log 0 = 0,
 * which is also the data log-likelihood gained by fitting that single
 * coupling with every other parameter fixed (max over d of
 * d f - log(1 - p + p e^d)).  Reading: the paper points to the literature
 * for "the most distant" criterion; this is the one used here.  +inf where
 * f > 0 = p or f < 1 = p.  Every element is scored, active or not (the
 * paper selects among all quadruplets). */
void orc_activation_scores(const double *fij, const double *pij, int L, int q, double *score)
{
    const size_t n = orc_n_elements(L, q);
    for (size_t e = 0; e < n; ++e) {
        int i, j, a, b;
        orc_element(e, L, q, &i, &j, &a, &b);
        const size_t x = jidx(L, q, i, j, a, b);
        const double f = fij[x], p = pij[x];
        double A = 0.0;
        if (f > 0.0) A += (p > 0.0) ? f * log(f / p) : INFINITY;
        if (f < 1.0) A += (p < 1.0) ? (1.0 - f) * log((1.0 - f) / (1.0 - p)) : INFINITY;
        score[e] = A > 0.0 ? A : 0.0;
    }
}

typedef struct {
    double s;
    size_t e;
} orc_scored;

static int orc_cmp_asc(const void *x, const void *y)
{
    const orc_scored *u = (const orc_scored *)x, *v = (const orc_scored *)y;
    if (u->s < v->s) return -1;
    if (u->s > v->s) return 1;
    return u->e < v->e ? -1 : (u->e > v->e ? 1 : 0);
}

static int orc_cmp_desc(const void *x, const void *y)
{
    const orc_scored *u = (const orc_scored *)x, *v = (const orc_scored *)y;
    if (u->s > v->s) return -1;
    if (u->s < v->s) return 1;
    return u->e < v->e ? -1 : (u->e > v->e ? 1 : 0);
}

/* Remove the n active elements with the smallest decimation score (ties:
 * lower element number first): active = 0 and J = 0 at both (i,j,a,b) and
 * (j,i,b,a).  Returns the number removed (n, capped at the active count). */
long orc_graph_decimate(double *J, uint8_t *active, const double *score, int L, int q, long n)
{
    const size_t ne = orc_n_elements(L, q);
    orc_scored *c = (orc_scored *)malloc((ne ? ne : 1) * sizeof(orc_scored));
    size_t m = 0;
    for (size_t e = 0; e < ne; ++e) {
        int i, j, a, b;
        orc_element(e, L, q, &i, &j, &a, &b);
        if (active[jidx(L, q, i, j, a, b)]) {
            c[m].s = score[e];
            c[m].e = e;
            ++m;
        }
    }
    qsort(c, m, sizeof(orc_scored), orc_cmp_asc);
    long done = 0;
    for (size_t k = 0; k < m && done < n; ++k, ++done) {
        int i, j, a, b;
        orc_element(c[k].e, L, q, &i, &j, &a, &b);
        active[jidx(L, q, i, j, a, b)] = active[jidx(L, q, j, i, b, a)] = 0;
        J[jidx(L, q, i, j, a, b)] = J[jidx(L, q, j, i, b, a)] = 0.0;
    }
    free(c);
    return done;
}

/* Select the n elements with the largest activation score among all
 * elements (ties: lower element number first) and make them active in both
 * halves; elements already active stay so.  Returns how many were newly
 * activated. */
long orc_graph_activate(uint8_t *active, const double *score, int L, int q, long n)
{
    const size_t ne = orc_n_elements(L, q);
    orc_scored *c = (orc_scored *)malloc((ne ? ne : 1) * sizeof(orc_scored));
    for (size_t e = 0; e < ne; ++e) {
        c[e].s = score[e];
        c[e].e = e;
    }
    qsort(c, ne, sizeof(orc_scored), orc_cmp_desc);
    long fresh = 0;
    for (size_t k = 0; k < ne && (long)k < n; ++k) {
        int i, j, a, b;
        orc_element(c[k].e, L, q, &i, &j, &a, &b);
        if (!active[jidx(L, q, i, j, a, b)]) ++fresh;
        active[jidx(L, q, i, j, a, b)] = active[jidx(L, q, j, i, b, a)] = 1;
    }
    free(c);
    return fresh;
}

/* Eq. 5 on a sparse graph: as orc_update, then every inactive coupling
 * element is zero (inactive couplings are not parameters of the model). */
void orc_update_masked(double *h, double *J, const double *fi, const double *fij, const int32_t *C,
                       int M, double lr, int L, int q, const uint8_t *active)
{
    orc_update(h, J, fi, fij, C, M, lr, L, q);
    for (size_t x = 0; x < (size_t)L * L * q * q; ++x)
        if (!active[x]) J[x] = 0.0;
}
