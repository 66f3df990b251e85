/*
 * bmdca.h -- C ABI of libbmdca.so, the GB300 (sm_103a) hot path of
 * Boltzmann-machine Direct Coupling Analysis (bmDCA) as described in
 * adabmDCA 2.0 (Muntoni, Pagnani, Weigt, Zamponi et al., arXiv 2501.18456).
 *
 * Model (Sec. 2.1, Eq. 1): a Potts model over L sites and q symbols,
 *     p(s) = exp(-E(s)) / Z,
 *     E(s) = - sum_i h_i(s_i) - sum_{i<j} J_ij(s_i, s_j),
 * with J_ij(a,b) = J_ji(b,a) and J_ii = 0.  Symbol 0 is the alignment gap
 * (Sec. 2.3, Table 1).
 *
 * Common conventions for every entry point:
 *   - Layouts are C row-major.  h is float[L][q]; J is float[L][L][q][q]
 *     with J[i][j][a][b] = J_ij(a,b).  Sequences and chain states are
 *     uint8[n][L], every symbol < q.
 *   - Pair counts use the upper block triangle: for i <= j the q x q block
 *     (i,j) sits at block index i*L - i*(i-1)/2 + (j-i) and holds
 *     C[a][b] = #{chains m : s_i = a, s_j = b}.  There are L*(L+1)/2
 *     blocks; the diagonal block (i,i) carries the single-site counts on
 *     its diagonal.
 *   - `where` arguments: BM_HOST (0) for a host pointer, BM_DEVICE (1) for
 *     a device pointer on the current device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is stream-ordered and asynchronous, except the
 *     ones that return a host scalar (they synchronise the stream) and the
 *     ones that copy from/to pageable host memory.
 *   - The caller owns every raw buffer it passes.  The library owns the
 *     internals of bm_model / bm_chains handles (device memory included)
 *     until the matching *_free call.
 *   - Return value: BM_OK or a negative bm_status.  No exception crosses
 *     the ABI.  bm_last_error() returns a message for the calling thread's
 *     last failure.  Invalid arguments are rejected before any GPU work.
 *   - Limits: 1 <= q <= 32, 1 <= L <= 4096, M >= 1.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 *     Work on one handle must also not overlap across streams: a handle's
 *     scratch (derived coupling layouts, the chain counts' one-hot operand,
 *     split-tile partials and tickets, the graph selection keys) is reused
 *     by every call, so calls on different streams need the caller's
 *     ordering (an event) between them.
 *
 * Random numbers: every draw uses Philox4x64-10 (Salmon et al., SC'11) with
 * key (seed, 0) and counter (chain, sweep, site, tag), tag 0 for Gibbs
 * draws, tag 1 for chain initialisation, tags 2 and 3 for the Metropolis
 * proposal and acceptance (bm_model_set_sampler); the uniform is the top 24 bits
 * of output word 0 scaled by 2^-24.  Results therefore depend only on the
 * seed and the global chain / sweep / site indices, not on launch shapes.
 */
#ifndef BMDCA_H
#define BMDCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bm_model_s *bm_model;    /* device h, J and derived layouts */
typedef struct bm_chains_s *bm_chains;  /* device chain states + seed + sweep counter */

typedef enum {
    BM_OK = 0,
    BM_EINVAL = -1,    /* bad argument, shape, symbol or asymmetric J */
    BM_ENOMEM = -2,    /* device allocation failed */
    BM_ECUDA = -3,     /* a CUDA runtime call failed (message has the name) */
    BM_ENUMERIC = -4,  /* NaN/Inf in parameters */
    BM_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    BM_EDEVICE = -6,   /* a device-side check recorded an error */
    BM_EBUSY = -7      /* resource in use */
} bm_status;

enum { BM_HOST = 0, BM_DEVICE = 1 };

/* Which kernel form bm_gibbs_sweep uses (bm_model_set_engine). */
enum {
    BM_ENGINE_SIMT = 0,  /* FP32 CUDA-core gather of J rows */
    BM_ENGINE_AUTO = 1,  /* default: the measured faster form.  The two-CTA form when
                            4 <= q <= 8, L >= 120, M >= 4096 and a site block's 64-column
                            K chunks number at most 3x its sites (there it takes its
                            tensor-memory operand form).  Otherwise tensor cores when
                            M*L^2 >= T(q) and L >= L0(q) (q >= 16: 2e7, 48; q 10-15: 5e7,
                            100; q 8-9: 2.5e8, 120; q 5-7: 5e8, 180; q 2-4: 5e7, 150) and
                            the shape fits, else CUDA cores.  Among the tensor-core forms
                            the two-CTA one for long block pairs (L*q^2 >= 98000 with more
                            than 96 chains per cluster, >= 63000 otherwise) when it needs
                            no more waves of CTAs than the one-CTA form. */
    BM_ENGINE_MMA = 2,   /* tensor cores: one-hot x (fp16 hi + fp16 lo) J, FP32 accumulate;
                            one CTA per SM computes both blocks of a block pair */
    BM_ENGINE_MMA_PAIR = 3  /* the same arithmetic split over the two CTAs of a cluster: each
                               CTA streams and redraws every other site block, the new states
                               are exchanged through distributed shared memory.  Where a
                               block's K chunks number at most 4x its sites, the one-hot
                               states are the MMA's A operand in tensor memory (128 chains
                               per cluster, one per TMEM lane) and J the B operand */,
    BM_ENGINE_MMA_PAIR2 = 4 /* the two-CTA form with the two SMs' tensor cores paired
                               (tcgen05 cta_group::2): one MMA of M = 256 rows covers both
                               CTAs' site blocks, and each CTA generates and holds the
                               one-hot rows of half of the cluster's chains */
};

/* Library version string, e.g. "bmdca-gb300 0.1". */
const char *bm_version(void);

/* Message for the calling thread's most recent failure ("" if none). */
const char *bm_last_error(void);

/*
 * bm_potts_load -- upload a Potts model (Eq. 1) and build its device layouts.
 *   h     : float[L][q] fields.
 *   J     : float[L][L][q][q] couplings, J[i][j][a][b] = J_ij(a,b).
 *   where : BM_HOST or BM_DEVICE for both h and J (copied, not retained).
 * Checks (BM_EINVAL): L, q in range; J exactly symmetric
 * (J[i][j][a][b] == J[j][i][b][a]); J[i][i] == 0.  NaN/Inf -> BM_ENUMERIC.
 * Synchronises `stream` (the checks are read back).  *out receives the
 * handle on success.
 */
int bm_potts_load(const float *h, const float *J, int L, int q, int where, void *stream,
                  bm_model *out);

/* Release a model and its device memory.  NULL is accepted. */
int bm_potts_free(bm_model m);

/* Copy the current parameters (after any bm_update) to h / J (either may be
 * NULL), same layouts as bm_potts_load.  Stream-ordered. */
int bm_potts_get(bm_model m, float *h, float *J, int where, void *stream);

/* Overwrite the live parameters of m in place from h / J (either may be
 * NULL; same layouts as bm_potts_load).  No symmetry or finiteness check:
 * the caller guarantees the invariants bm_potts_load verifies (use it for
 * parameters that came out of this library, e.g. a checkpoint).  Allocates
 * nothing; stream-ordered. */
int bm_potts_set(bm_model m, const float *h, const float *J, int where, void *stream);

/* Synchronise `stream` and report device-side errors recorded by earlier
 * kernels of this model, then clear them: BM_OK; BM_ETIMEOUT (a bounded
 * wait gave up); BM_EINVAL (a scored sequence held a symbol >= q);
 * BM_ENUMERIC (a coupling beyond the fp16 range, |J| > 65504, reached the
 * fp16 split layout of the tensor-core sweep or fields: it was clamped and
 * those results are invalid; the FP32 engine has no such limit).  bm_update
 * with a Pearson request performs the timeout check. */
int bm_device_status(bm_model m, void *stream);

/* L and q of a model. */
int bm_potts_shape(bm_model m, int *L, int *q);

/*
 * bm_chains_init -- create M persistent chains (Sec. 2.1, PCD) for model m.
 *   init_or_null : uint8[M][L] start states (`where` says host/device), or
 *                  NULL for uniformly random states: symbol of chain m at
 *                  site i = floor(u24 * q / 2^24), u24 from Philox counter
 *                  (m, 0, i, 1).
 *   seed         : Philox key word 0 for every later draw of these chains.
 * The sweep counter starts at 0.  Symbols >= q in init -> BM_EINVAL
 * (checked on the device; the call synchronises `stream`).
 */
int bm_chains_init(bm_model m, int M, uint64_t seed, const uint8_t *init_or_null, int where,
                   void *stream, bm_chains *out);

/*
 * bm_chains_init_shard -- chains chain0 .. chain0+M-1 of a larger ensemble
 * (one shard per GPU when the chains are split across devices, Sec. 2.1:
 * chains are independent).  Uniformly random start as above with the
 * GLOBAL chain index in every Philox counter, so the shards of an ensemble
 * draw exactly the states of one handle holding all of it: the counts of
 * the shards sum to its counts.  The handle keeps chain0 for its sweeps.
 */
int bm_chains_init_shard(bm_model m, int M, uint64_t seed, uint64_t chain0, void *stream, bm_chains *out);

/* Release chains.  NULL is accepted. */
int bm_chains_free(bm_chains c);

/* Copy the chain states (uint8[M][L]) to dst.  Stream-ordered. */
int bm_chains_get(bm_chains c, uint8_t *dst, int where, void *stream);

/* Overwrite the chain states from src (uint8[M][L]); the sweep counter is
 * left unchanged.  Symbols are not re-checked (caller guarantees < q). */
int bm_chains_set(bm_chains c, const uint8_t *src, int where, void *stream);

/* Read / set the global sweep counter (the Philox `sweep` word of the next
 * sweep).  Setting it lets a caller replay or resume a run bit-identically. */
int bm_chains_sweep_counter(bm_chains c, uint64_t *sweep);
int bm_chains_set_sweep_counter(bm_chains c, uint64_t sweep);
int bm_chains_shape(bm_chains c, int *M, int *L);

/*
 * bm_gibbs_sweep -- nsweeps persistent-chain Gibbs sweeps (Sec. 2.1,
 * "Monte Carlo estimation of the gradient"; a sweep proposes every site
 * once, Sec. 3.3).  Sites are visited in order i = 0..L-1.  For chain m
 * and site i the local field H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j) is
 * formed from the current states, and s_i is drawn from p(a) ~
 * exp(beta * H_i(a)) by inverse CDF (first a with u * S_total < S_a over
 * prefix sums in a ascending, weights exp(beta*H_a - max_b beta*H_b)) with
 * u from Philox counter (m, sweep, i, 0).  The sweep counter advances by
 * nsweeps.  beta = 1 for training; beta != 1 samples p ~ exp(-beta E)
 * (Sec. 4.1 sampling at inverse temperature).  nsweeps >= 0, beta finite.
 */
int bm_gibbs_sweep(bm_model m, bm_chains c, int nsweeps, float beta, void *stream);

/* Select the kernel form used by bm_gibbs_sweep for this model
 * (BM_ENGINE_*).  BM_EINVAL for an unknown engine. */
int bm_model_set_engine(bm_model m, int engine);

/* Update rule of the sweeps (Sec. 2.1: the chains are updated by Gibbs or
 * Metropolis-Hastings steps; the --sampler option of the training and
 * sampling commands). */
enum { BM_SAMPLER_GIBBS = 0, BM_SAMPLER_METROPOLIS = 1 };

/*
 * bm_model_set_sampler -- the update applied at each site by bm_gibbs_sweep,
 * the batch sweeps and the server's sampling requests for this model.
 *   BM_SAMPLER_GIBBS (default): s_i redrawn from the conditional (above).
 *   BM_SAMPLER_METROPOLIS: one Metropolis-Hastings step per site, sites in
 *     order 0..L-1: proposal a' = k + (k >= s_i), k = floor(u_p (q-1)),
 *     uniform over the q-1 other symbols, u_p from Philox counter
 *     (m, sweep, i, 2); accepted iff u_a < exp(beta (H_i(a') - H_i(s_i)))
 *     (always when that difference is >= 0), u_a from counter (m, sweep, i,
 *     3), H_i the local field of the current states (FP32); q = 1 keeps
 *     the state.  All engines but the one-CTA form run it; with
 *     BM_ENGINE_MMA the two-CTA form is used instead.
 * BM_EINVAL for an unknown sampler.
 */
int bm_model_set_sampler(bm_model m, int sampler);

/* The kernel form bm_gibbs_sweep runs for this model and M chains, with
 * BM_ENGINE_AUTO resolved: BM_ENGINE_SIMT, BM_ENGINE_MMA,
 * BM_ENGINE_MMA_PAIR or BM_ENGINE_MMA_PAIR2, written to *engine_out.  BM_EINVAL for a NULL
 * argument or M < 1.  May query the device (cluster occupancy). */
int bm_model_sweep_engine(bm_model m, int M, int *engine_out);

/* Kernel form used by bm_chain_stats (bm_chains_set_stats_engine). */
enum {
    BM_STATS_AUTO = 0,      /* default: the fastest measured form (BM_STATS_MMA_FP8 when M < 2^24,
                               else BM_STATS_SIMT) */
    BM_STATS_SIMT = 1,      /* CUDA cores, shared-memory histograms */
    BM_STATS_MMA_BF16 = 2,  /* tensor cores, BF16 one-hot operands built in shared memory */
    BM_STATS_MMA_FP8 = 3    /* tensor cores (CTA pairs), FP8 E4M3 one-hot X^T written once to
                               device memory (L*q x M rounded up to 128 bytes) and streamed by
                               TMA; on first use the chains handle also allocates a workspace for
                               the partial counts of output tiles split along the chains
                               (64 KB x 4 x SMs/2, ~20 MB on 152 SMs, plus its tickets); both are
                               owned by the handle and freed with it */
};

/* Select the bm_chain_stats kernel form for these chains (all forms give
 * identical, exact counts; the tensor-core forms need M < 2^24 and fall back
 * to BM_STATS_SIMT otherwise).  BM_EINVAL for an unknown engine. */
int bm_chains_set_stats_engine(bm_chains c, int engine);

/* Synchronise `stream` and report device-side errors recorded by earlier
 * kernels on these chains (bounded waits that gave up): BM_OK or
 * BM_ETIMEOUT (the error word is then cleared). */
int bm_chains_device_status(bm_chains c, void *stream);

/*
 * bm_chain_stats -- model statistics from the chains (Sec. 2.1: p_i, p_ij
 * estimated as chain frequencies).  Writes int32 counts in the upper
 * block-triangle layout above to counts_dev (device, L*(L+1)/2*q*q
 * int32, fully overwritten).  p = count / M.  Exact (integer).
 */
int bm_chain_stats(bm_chains c, int32_t *counts_dev, void *stream);

/*
 * bm_seq_weights -- importance weights, Eq. 7: w_m = 1 / N_m where N_m is
 * the number of sequences n (m included) whose identity with m -- number
 * of positions with equal symbols, gap included -- is >= ceil(seqid * L)
 * (the ceiling taken after subtracting 1e-9, so seqid = 0.8, L = 120 gives
 * 96).  msa_dev: device uint8[N][L]; w_dev: device float[N];
 * meff_host (may be NULL): M_eff = sum_m w_m in FP64 (Sec. 3.3), returned
 * after synchronising `stream`.  0 < seqid <= 1.
 */
int bm_seq_weights(const uint8_t *msa_dev, int N, int L, double seqid, float *w_dev,
                   double *meff_host, void *stream);

/* Largest N accepted by bm_seq_weights_static (4 MiB of device memory). */
#define BM_SEQ_WEIGHTS_STATIC_MAX_N 1048576

/*
 * bm_seq_weights_static -- the same weights and M_eff as bm_seq_weights,
 * computed without allocating any device memory.  The paper has no
 * counterpart: this is a deployment variant for callers that must not
 * allocate, e.g. code running while another framework's caching allocator
 * holds the device memory, serving loops that must not enter the driver's
 * allocator (cudaMalloc/cudaFree may synchronise the device), or embedders
 * that give the library a fixed memory budget.
 *   Scratch: one file-scope device array of 256 B + 4 * MAX_N bytes, held
 *   on every GPU that loads the library until the process exits.
 *   N > BM_SEQ_WEIGHTS_STATIC_MAX_N -> BM_EINVAL (message names the limit).
 *   The first call on a device (with that device current) looks up the
 *   array's device address; make that first call before any stream capture.
 *   The address is kept for the life of the process: after cudaDeviceReset
 *   (which unloads the library's module with its array) this entry point
 *   must not be called again on that device in the same process.
 *   Every call reuses the same array (its counters are cleared at the start
 *   of each call), so calls whose GPU work overlaps -- different streams or
 *   host threads -- race and must be serialised by the caller.
 * Arguments, results and synchronisation are those of bm_seq_weights.
 */
int bm_seq_weights_static(const uint8_t *msa_dev, int N, int L, double seqid, float *w_dev,
                          double *meff_host, void *stream);

/*
 * bm_data_stats -- empirical frequencies, Eq. 3, with the pseudocount of
 * Eqs. 8-9:  f_i = (1-alpha) f_i^data + alpha/q,
 *            f_ij = (1-alpha) f_ij^data + alpha/q^2   (i != j),
 * f^data weighted by w (w_or_null == NULL: uniform weights) and divided by
 * M_eff = sum w.  pseudocount < 0 selects the paper's default alpha =
 * 1/M_eff (Sec. 3.3).  Outputs (device): fi_dev float[L][q], fij_dev
 * float[L][L][q][q] (diagonal blocks: fij[i][i][a][b] = delta_ab f_i(a)).
 * Weighted sums are accumulated exactly in 64-bit fixed point (2^-40
 * resolution per weight), so the result is deterministic.
 */
int bm_data_stats(const uint8_t *msa_dev, const float *w_or_null, int N, int L, int q,
                  double pseudocount, float *fi_dev, float *fij_dev, void *stream);

/*
 * bm_update -- one Boltzmann-learning step, Eq. 5:
 *     h_i(a)    += lr (f_i(a)    - p_i(a)),
 *     J_ij(a,b) += lr (f_ij(a,b) - p_ij(a,b))   (i != j; J_ii stays 0),
 * with p = counts / M (counts from bm_chain_stats, device) and f from
 * bm_data_stats (device).  In the same pass the Pearson correlation of the
 * connected correlations C^data = f_ij - f_i f_j and C^model = p_ij - p_i p_j
 * over i < j and all (a,b) is reduced in FP64 (Sec. 2.1, convergence
 * criterium).
 *   pearson_out == NULL : no Pearson, update applied, fully asynchronous.
 *   pearson_out != NULL : synchronises `stream`; *pearson_out = rho of the
 *                         statistics passed in (the parameters that
 *                         produced the chains); the update is applied only
 *                         if rho < target (pass target > 1 to always apply).
 *   applied_out (may be NULL) receives 1 if the parameters changed.
 */
int bm_update(bm_model m, const float *fi_data, const float *fij_data, const int32_t *counts,
              int M, float lr, double target, double *pearson_out, int *applied_out,
              void *stream);

/*
 * Sparse interaction graphs (Sec. 2.2, "Training sparse models").
 *
 * An element is one coupling entry J_ij(a,b) with i < j; its mirror J_ji(b,a)
 * follows it.  Elements are numbered pair by pair in row order, (0,1),
 * (0,2), ..., (1,2), ..., and within a pair a*q + b; ties in a selection go
 * to the lower number.  The graph is kept on the model as one activity byte
 * per entry of J's layout [i][j][a][b] (symmetric; diagonal blocks 0).  Once
 * a graph is enabled, bm_update writes inactive couplings as zero; the sweeps
 * and scores read J as usual.  bm_potts_set stores J as given, inactive
 * entries included, and does not change the graph; the next bm_update zeroes
 * the inactive couplings again.  Memory owned by the model: L*L*q*q bytes of
 * activity, 8 bytes per element of selection keys, a few KB more.
 */

/* Create the graph: dense != 0 makes every element active (J unchanged);
 * dense == 0 makes none active and zeroes every coupling.  May be called
 * again to reset.  BM_EINVAL for a NULL model; BM_ECUDA on allocation or
 * launch failure.  Asynchronous on `stream`. */
int bm_graph_enable(bm_model m, int dense, void *stream);

/* Drop the graph (the model is fully connected again; J is not changed). */
int bm_graph_disable(bm_model m);

/* Active elements and all elements (L(L-1)/2 q^2); density = ratio.  A model
 * without a graph counts every element as active. */
int bm_graph_count(bm_model m, long long *n_active, long long *n_elements);

/* Copy the activity bytes [L][L][q][q] to active_out (BM_HOST or BM_DEVICE;
 * a host copy synchronises `stream`).  BM_EINVAL without a graph. */
int bm_graph_get(bm_model m, uint8_t *active_out, int where, void *stream);

/*
 * bm_graph_decimate -- edDCA graph step: remove the n active elements (n is
 * capped at the active count) whose removal perturbs the model least, scored
 * by the symmetric Kullback-Leibler divergence between the model and the
 * model without the element,
 *     D = J (p - p'),   p' = p e^{-J} / (1 - p + p e^{-J}),
 * p = counts / M the chains' pair frequency of the element (FP64; negative
 * rounding taken as 0).  Removed elements become inactive and both coupling
 * entries become 0.  counts_dev: bm_chain_stats output of the chains sampled
 * from this model.  *removed_out = the number removed.  Synchronises
 * `stream`.  BM_EINVAL: NULL argument, no graph, M < 1 or n < 0.
 */
int bm_graph_decimate(bm_model m, const int32_t *counts_dev, int M, long long n, long long *removed_out,
                      void *stream);

/*
 * bm_graph_activate -- eaDCA graph step: among all elements select the n
 * (capped at the element count) whose model pair frequency p = counts / M is
 * farthest from the data's f (fij_dev from bm_data_stats), scored by the
 * Bernoulli Kullback-Leibler divergence
 *     A = f log(f/p) + (1-f) log((1-f)/(1-p))   (0 log 0 = 0; +inf when
 *                                                p = 0 < f or f < 1 = p),
 * the likelihood gain of fitting that coupling alone (FP64).  Selected
 * elements become active (their couplings start at 0, the value they had);
 * elements already active stay so.  *activated_out = newly activated count.
 * Synchronises `stream`.  BM_EINVAL: NULL argument, no graph, M < 1, n < 0.
 */
int bm_graph_activate(bm_model m, const float *fij_dev, const int32_t *counts_dev, int M, long long n,
                      long long *activated_out, void *stream);

/*
 * bm_energy_score -- DCA energy E(s) of n sequences (Eq. 1; Sec. 4.3: low
 * energy = good sequence).  seqs_dev: device uint8[n][L]; E_dev: device
 * float[n].  FP32 accumulation (large batches, n*L >= 3.3e6, stream J
 * through shared memory; the sum order, and so the last bits, differ
 * between the two forms).  A symbol >= q is flagged: the next
 * bm_device_status returns BM_EINVAL and that sequence's energy is
 * unspecified.
 */
int bm_energy_score(bm_model m, const uint8_t *seqs_dev, int n, float *E_dev, void *stream);

/*
 * bm_mutant_scan -- single-mutant library (Sec. 4.4): dE[i][a] =
 * E(wt with s_i = a) - E(wt) = -(H_i(a) - H_i(wt_i)) with H the local
 * field at the wild type; dE[i][wt_i] = 0.  wt: uint8[L] (`where`);
 * dE_dev: device float[L][q].
 */
int bm_mutant_scan(bm_model m, const uint8_t *wt, int where, float *dE_dev, void *stream);

/* Numerical form of bm_fields. */
enum {
    BM_FIELDS_FP32 = 0,    /* CUDA cores: FP32 sum over j ascending */
    BM_FIELDS_FP16X2 = 1,  /* tensor cores: J = fp16 hi + fp16 lo (round to nearest), FP32
                              accumulation; the numerics of the tensor-core Gibbs sweep */
    BM_FIELDS_BF16X2 = 2   /* tensor cores: J = bf16 hi + bf16 lo, FP32 accumulation */
};

/*
 * bm_fields -- local fields of n sequences, H[k][i][a] = h_i(a) +
 * sum_{j != i} J_ij(a, s_j^k): the field whose softmax is the Gibbs
 * conditional of site i (Sec. 2.1) and from which single-mutant energies
 * are formed (Sec. 4.4).  seqs_dev: device uint8[n][L]; H_dev: device
 * float[n][L][q], fully written.  `form` is a BM_FIELDS_* value (BM_EINVAL
 * otherwise).  A symbol >= q contributes nothing; the next bm_device_status
 * then returns BM_EINVAL.  The tensor-core forms use stream-ordered scratch
 * of min(n, 65536) * Kp * 2 bytes (Kp = L*q rounded up to 64) and rebuild
 * their split copy of J after a parameter change (bm_potts_set, an applied
 * bm_update).
 */
int bm_fields(bm_model m, const uint8_t *seqs_dev, int n, float *H_dev, int form, void *stream);

/*
 * Batched sweeps of many independent models (uneven-L training of many
 * models on one GPU).  A batch groups (model, chains) pairs with the same q;
 * bm_batch_sweep runs nsweeps sweeps of every pair in ONE launch over a work
 * list of chain tiles, longest models first.  Two forms:
 *  - tensor cores, when q >= 2, no model's engine is BM_ENGINE_SIMT and
 *    every model fits: the two-CTA sweep, one
 *    cluster per (model, tile), each cluster reading its model's arguments
 *    and TMA descriptor from the list (refreshed from host memory by each
 *    call); the arithmetic per chain is that of BM_ENGINE_MMA_PAIR;
 *  - otherwise CUDA cores, replayed from a captured CUDA graph that first
 *    refreshes the list (current parameter pointers, sweep counters); the
 *    states drawn equal those of bm_gibbs_sweep with BM_ENGINE_SIMT on each
 *    pair separately (same Philox uniforms, same FP32 summation order).
 * The handles stay owned by the caller and must outlive the batch; chains
 * sweep counters advance.
 */
typedef struct bm_batch_s *bm_batch;

/* BM_EINVAL: empty batch, mismatched chains, different q, or L too large
 * for shared memory. */
int bm_batch_create(const bm_model *models, const bm_chains *chains, int count, bm_batch *out);
int bm_batch_free(bm_batch b);

/* Times every fitting tile shape (CUDA cores: chains per CTA x pipeline
 * stages; tensor cores: the cap on chains per cluster) on scratch copies of
 * the states (the chains do not move) and keeps the fastest.  Synchronises
 * `stream`. */
int bm_batch_autotune(bm_batch b, void *stream);

/* nsweeps sweeps at inverse temperature beta of every pair (one graph
 * launch on `stream`). */
int bm_batch_sweep(bm_batch b, int nsweeps, float beta, void *stream);

/* Current tile shape: chains per CTA (per cluster in the tensor-core form),
 * pipeline stages (one-hot ring slots in the tensor-core form), CTAs per
 * launch. */
int bm_batch_shape(bm_batch b, int *chains_per_cta, int *stages, int *ctas);

/*
 * Serving with continuous batching (Sec. 4.1 sampling, Sec. 4.3 scoring,
 * Sec. 4.4 single-mutant scans of trained models).
 *
 * A server keeps models resident and runs requests on a pool of CUDA
 * streams from a worker thread.  Requests wait in arrival order; whenever a
 * stream is free and the request's device scratch fits in the memory budget
 * beside the requests already running, it is admitted (a later request that
 * fits may start before an earlier one that does not), so work that arrives
 * while other requests run joins them on the device as slots and memory
 * free up.  Each request's result depends only on the request itself
 * (sampling uses the request's own Philox key), so it is the same alone and
 * in any mix.
 *
 * Host buffers (in / out) are owned by the caller and must stay valid until
 * the request completes; pinned memory lets copies overlap other work
 * (device pointers are accepted too).  Models must not be freed or have
 * their parameters changed while the server holds them.  All bm_server_*
 * calls are thread-safe.
 */
typedef struct bm_server_s *bm_server;

enum {
    BM_REQ_SAMPLE = 1,  /* n chains from uniform random states (Philox key `seed`, tag 1),
                           nsweeps Gibbs sweeps at beta (draws keyed by `seed`, tag 0);
                           out: uint8[n][L] final states.  Scratch n*L bytes. */
    BM_REQ_SCORE = 2,   /* energies of n sequences, in: uint8[n][L]; out: float[n].
                           Scratch n*(L+4) bytes. */
    BM_REQ_SCAN = 3     /* single-mutant scan of the wild type in: uint8[L];
                           out: float[L][q] (bm_mutant_scan).  Scratch L*(4q+1) bytes. */
};

typedef struct {
    int type;         /* BM_REQ_* */
    int model;        /* index returned by bm_server_add_model */
    int n;            /* SAMPLE, SCORE: number of sequences (>= 1) */
    int nsweeps;      /* SAMPLE: >= 0 */
    float beta;       /* SAMPLE: finite */
    uint64_t seed;    /* SAMPLE: Philox key of the request */
    const void *in;   /* SCORE: uint8[n][L]; SCAN: uint8[L]; else unused */
    void *out;        /* see BM_REQ_* */
} bm_request;

typedef struct {
    long long submitted, completed, failed;
    double p50_ms, p99_ms, mean_ms;  /* latency (submit to completion seen by the worker) */
    double sequences;                /* SAMPLE n + SCORE n + SCAN L*q over completed requests */
    double span_s;                   /* first submit to last completion */
    int max_running;                 /* most requests on the device at once */
} bm_server_stats;

/* New server on the current device: `budget_bytes` of device scratch for
 * running requests, `slots` streams (1..256).  BM_EINVAL / BM_ENOMEM. */
int bm_server_create(size_t budget_bytes, int slots, bm_server *out);

/* Drains (waits for every submitted request) and frees the server.  The
 * models stay with the caller. */
int bm_server_destroy(bm_server s);

/* Makes a model resident; prepares its tensor-core layout (synchronously)
 * so requests never rebuild it.  *id receives the model's index. */
int bm_server_add_model(bm_server s, bm_model m, int *id);

/* Queues a request (copied; the buffers are not).  *id receives its id.
 * BM_EINVAL for a malformed request, BM_ENOMEM if its scratch alone
 * exceeds the budget. */
int bm_server_submit(bm_server s, const bm_request *r, uint64_t *id);

/* Blocks until request `id` completes (timeout_ms < 0: no limit);
 * *status receives its outcome (BM_OK or an error code), *latency_ms its
 * latency.  BM_ETIMEOUT if it did not complete in time; BM_EINVAL for an
 * unknown or already waited id. */
int bm_server_wait(bm_server s, uint64_t id, double timeout_ms, int *status, double *latency_ms);

/* Counters and latency percentiles of the requests completed so far;
 * reset = 1 clears them afterwards. */
int bm_server_stats_get(bm_server s, bm_server_stats *out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* BMDCA_H */
