/*
 * madflow_gb300.h -- C ABI of the GB300 (sm_103a) event-parallel Monte Carlo
 * hot path of MadFlow (arXiv:2211.14056, "Extending MadFlow: device-specific
 * optimization").
 *
 * What the library computes, in the paper's terms:
 *   - Sec. 1: a tensorised Vegas integration whose events are all independent
 *     ("parallelized in the event axis", abstract);
 *   - Sec. 2: the per-event tree-level matrix element of an autogenerated
 *     process, which the paper moves into a device-specific custom operator
 *     built from "vertices, spinors or propagators", here one fused kernel per
 *     process with no per-diagram tensor in device memory (the memory-footprint
 *     point of Sec. 2 and of Table 1's diagram counts 36 / 267);
 *   - Sec. 2 (end): the derivative of that operator, which the paper leaves out.
 *
 * Conventions shared by every call:
 *   - units GeV, cross sections in pb;
 *   - particle order: the two incoming partons, t, tbar, then the final light
 *     partons (gluons first);
 *   - momenta arrays are structure-of-arrays FP64: element (particle i,
 *     component c, event e) at [(i*4 + c)*n + e], components (E, px, py, pz),
 *     partonic centre-of-mass frame, beam 1 along +z;
 *   - ownership: every device buffer is allocated and owned by the caller;
 *     handles (mf_process, mf_grid) are owned by the library and freed by the
 *     matching destroy call; device scratch is allocated when a handle is
 *     created, never inside a compute call;
 *   - streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Calls are asynchronous on it, except those with host
 *     outputs, which synchronise that stream before returning;
 *   - errors: a negative status is an error, a positive one a warning; the
 *     message of the last failing call on this thread is mf_last_error().  No
 *     C++ exception crosses this boundary.  On an error nothing has been
 *     launched unless the status is MF_ERR_CUDA.
 */
#ifndef MADFLOW_GB300_H
#define MADFLOW_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int mf_status;
#define MF_OK 0
#define MF_ERR_ARG (-1)         /* invalid argument, size or pointer */
#define MF_ERR_CUDA (-2)        /* a CUDA runtime call failed (message has the CUDA error) */
#define MF_ERR_UNSUPPORTED (-3) /* process / precision not built */
#define MF_ERR_COLOUR (-4)      /* colour matrix: wrong size, not symmetric, not the process's, not TF32-exact */
#define MF_ERR_TIMEOUT (-5)     /* reserved for a bounded device wait that gives up; no kernel of this
                                   library spins on a flag, so no entry point returns it */
#define MF_WARN_NEWTON 1        /* some events missed the massive-rescaling Newton tolerance; their weight is 0 */
#define MF_WARN_CAPACITY 2      /* more events were kept than the output buffers hold (mf_unweight) */

/* processes (gluon count of the colour-ordered recursion in brackets) */
#define MF_PROC_GG_TTX 1   /* g g -> t tbar        [2 gluons; 3 diagrams, 2 colour flows, 16 helicities]  */
#define MF_PROC_GG_TTXG 2  /* g g -> t tbar g      [3; 16 diagrams, 6 flows, 32 helicities]               */
#define MF_PROC_GG_TTXGG 3 /* g g -> t tbar g g    [4; 123 diagrams, 24 flows, 64 helicities]             */
/* u ubar -> t tbar g g: two quark lines, 38 Feynman diagrams decomposed onto
 * 12 colour structures (T^A)_{t u}(T^B)_{ubar tbar}, (T^A)_{t tbar}(T^B)_{ubar u}
 * over the ordered splits (A, B) of the two gluons; 64 helicities.  The same
 * phase space as g g -> t tbar g g (the synthetic luminosity serves u and
 * ubar); average 1/36.  Not covered: MF_FP32_TC, mf_grad and
 * mf_vegas_accumulate_static (MF_ERR_UNSUPPORTED). */
#define MF_PROC_UUX_TTXGG 4
/* e+ e- -> mu+ mu-: QED, one s-channel photon diagram (Feynman gauge),
 * massless leptons, 16 helicities, average 1/4, no colour (n_flow = 1, the
 * 1 x 1 matrix 1).  Fixed partonic energy only (lumi = 0), no cuts apply (no
 * final gluons); coupling e_qed.  Not covered: MF_FP32_TC, mf_grad and
 * mf_vegas_accumulate_static (MF_ERR_UNSUPPORTED). */
#define MF_PROC_EE_MUMU 5
/* The other subprocesses of p p -> t tbar g g (arXiv:2211.14056 Table 1:
 * pp -> t tbar g g sums them), crossings of the u ubar -> t tbar g g amplitude
 * (same 12-structure colour matrix, same restrictions; the u quark stands for
 * any light flavour, whose |M|^2 is the same: the channel's parton pairs in
 * the luminosity sum the flavours).  Final light partons: the gluon first,
 * then the (anti)quark; the cuts apply to both.
 *   MF_PROC_UXU_TTXGG   ubar u -> t tbar g g   (quark from beam 2; average 1/36, 1/2!)
 *   MF_PROC_UG_TTXGU    u g -> t tbar g u      (average 1/96)
 *   MF_PROC_GU_TTXGU    g u -> t tbar g u
 *   MF_PROC_UXG_TTXGUX  ubar g -> t tbar g ubar
 *   MF_PROC_GUX_TTXGUX  g ubar -> t tbar g ubar */
#define MF_PROC_UXU_TTXGG 6
#define MF_PROC_UG_TTXGU 7
#define MF_PROC_GU_TTXGU 8
#define MF_PROC_UXG_TTXGUX 9
#define MF_PROC_GUX_TTXGUX 10

/* arithmetic of the matrix element */
#define MF_FP64 0      /* everything in FP64 */
#define MF_FP32 1      /* amplitudes and colour sum in FP32 (FMA); sampling, Newton and sums FP64 */
#define MF_FP32_TC 2   /* FP32 amplitudes; colour sum J^T (D C) J with the integer matrix D C on the
                          tensor cores (mma.m16n8k8 TF32, J split into TF32 hi + lo, FP32 accumulate) */

typedef struct mf_process mf_process;
typedef struct mf_grid mf_grid;
typedef struct mf_pdf mf_pdf;

/* Process description (arXiv:2211.14056 Sec. 2: the process-dependent
 * functions a generator produces; here the parameters of a built kernel). */
typedef struct {
  int process_id;              /* MF_PROC_* */
  int n_ext;                   /* external particles: 4, 5 or 6, must match the process */
  const double* masses;        /* host [n_ext] GeV: 0, 0, m_t, m_t, 0...; the two top masses must agree;
                                  all 0 for MF_PROC_EE_MUMU */
  double top_width;            /* Gamma_t >= 0 in the internal top propagators */
  double g_s;                  /* strong coupling (fixed, no running) */
  int n_flow;                  /* colour flows: (n_ext-2)! for g g processes, 12 for u ubar -> t tbar g g */
  const int64_t* colour_num;   /* host [n_flow*n_flow] integer numerators of the process's colour matrix */
  int64_t colour_den;          /* common denominator; C = colour_num / colour_den */
  double sqrt_s;               /* hadronic sqrt(S) if lumi = 1, else the fixed partonic sqrt(s) */
  int lumi;                    /* 0: fixed partonic energy; 1: synthetic gluon luminosity;
                                  2: tabulated parton densities (pdf, pairs, mu_f below) */
  double lumi_N, lumi_a, lumi_b;  /* f(x) = N x^a (1-x)^b per gluon */
  double pt_cut_g;             /* final-gluon pT threshold (0 disables) */
  double dr_cut_gg;            /* final-gluon pair Delta R threshold (0 disables) */
  int precision;               /* MF_FP64, MF_FP32 or MF_FP32_TC */
  double e_qed;                /* electromagnetic coupling e = sqrt(4 pi alpha) (MF_PROC_EE_MUMU only) */
  /* lumi = 2 (tabulated parton densities): */
  const mf_pdf* pdf;           /* the set (mf_pdf_create); must outlive the process */
  int n_pairs;                 /* 1..8 parton pairs of the channel */
  const int* pairs;            /* host [n_pairs][2]: flavour indices (beam 1, beam 2) into the set */
  double mu_f;                 /* factorisation scale Q = mu_f * sqrt(s_hat) (> 0) */
} mf_process_desc;

/* Result of one Vegas iteration and of the combination of every iteration
 * recorded on the grid so far (Lepage's inverse-variance combination). */
typedef struct {
  double I_k, sigma_k;         /* this iteration: estimate and its error (pb) */
  double I, sigma, chi2dof;    /* combination over the grid's recorded iterations */
  int64_t n_events;            /* events of this iteration */
  int64_t n_pass;              /* events that passed the cuts (|M|^2 evaluated) */
  int64_t n_newton_fail;       /* events whose rescaling Newton missed its tolerance */
  int iterations;              /* iterations recorded on the grid */
} mf_result;

/* Create a process: validates the description (sizes, masses, colour
 * matrix against the library's exact trace-basis matrix), selects the built
 * kernel and sizes its launch from the device's occupancy.  *out is owned by
 * the library.  Errors: MF_ERR_ARG, MF_ERR_UNSUPPORTED, MF_ERR_COLOUR, MF_ERR_CUDA. */
mf_status mf_init_process(const mf_process_desc* desc, mf_process** out);
mf_status mf_destroy_process(mf_process* proc);

/* Vegas dimension of a process: 3 n_final - 4, plus 2 with the luminosity map. */
mf_status mf_process_ndim(const mf_process* proc, int* ndim);

/* Override the persistent launch: CTAs per SM for the fused and matrix-element
 * kernels (0 restores the occupancy-derived default).  Used by the autotuner
 * (arXiv:2211.14056 Sec. 3, Fig. 3: the block configuration matters). */
mf_status mf_set_ctas_per_sm(mf_process* proc, int ctas_per_sm);

/* Launch shape of the |M|^2 kernel of the iteration (arXiv:2211.14056 Sec. 3,
 * Fig. 3: the run time of 10^6 g g -> t t~ g g events depends on the threads
 * per block): warps_per_cta in 1..7 (32 to 224 threads per block; every warp
 * holds ~29 KB of shared memory, so 7 warps is the largest CTA that fits an
 * SM), 0 restores the default of 4.  Together with mf_set_ctas_per_sm it
 * spans the launch shapes of the launch-shape study; results do not depend on
 * it (the same per-warp code; only the order of the CTA partial sums).
 * *max_ctas_per_sm (host, may be NULL) receives how many such CTAs fit on
 * one SM at 50 bins per dimension (the occupancy limit of mf_set_ctas_per_sm).
 * Covers MF_PROC_GG_TTXGG with MF_FP32 or MF_FP32_TC (else
 * MF_ERR_UNSUPPORTED); MF_ERR_ARG outside [0, 7]. */
mf_status mf_set_launch_shape(mf_process* proc, int warps_per_cta, int* max_ctas_per_sm);

/* Tabulated parton densities (arXiv:2211.14056 Sec. 1: the integrand's
 * densities come from PDFFlow, a GPU interpolation of tabulated LHAPDF sets).
 * mf_pdf_create loads a set: xf host [nflav][nq][nx] = x f(x, Q^2) of each
 * flavour on nodes uniform in ln x (x_min .. x_max <= 1, nx nodes) and in
 * ln Q^2 (q2_min .. q2_max, nq nodes), 4 <= nq, nx <= 4096, 1 <= nflav <= 64.
 * The interpolation is log-bicubic Hermite: node slopes in ln x from finite
 * differences (mean of the neighbouring quotients, one-sided at the ends),
 * cubic Hermite in ln x on the rows around Q^2, then cubic Hermite in ln Q^2
 * with slopes from the same finite differences of those rows; queries outside
 * the table are clamped to its edge.  The set is copied to the device in FP64
 * and FP32 (allocated here, owned by the handle); MF_ERR_ARG on bad sizes,
 * ranges or non-finite values.
 * mf_pdf_eval: x f of flavour `flavour` at n points, x and q2 device [n] FP64
 * (inputs), xf device [n] FP64 (output), arithmetic in MF_FP64 or MF_FP32;
 * asynchronous on `stream`. */
mf_status mf_pdf_create(int nflav, int nq, int nx, double x_min, double x_max, double q2_min, double q2_max,
                        const double* xf, mf_pdf** out);
mf_status mf_pdf_destroy(mf_pdf* pdf);
mf_status mf_pdf_eval(const mf_pdf* pdf, int precision, int flavour, int64_t n, const double* x, const double* q2,
                      double* xf, void* stream);

/* Vegas grid (Lepage 1978, the integrator named in Sec. 1): nbins equal bins
 * per dimension (2 <= nbins <= 64), device edges [ndim][nbins+1], device
 * scratch for per-CTA partial sums sized for the process's largest launch,
 * and a host record of the iterations for the combination.  Owned by the
 * library. */
mf_status mf_grid_create(const mf_process* proc, int nbins, mf_grid** out);
mf_status mf_grid_destroy(mf_grid* grid);
/* Copy the edges to/from host memory [ndim*(nbins+1)] (checkpoint / resume);
 * these synchronise the device.  mf_grid_set checks that every row starts at
 * 0, ends at 1 and increases strictly. */
mf_status mf_grid_get(const mf_grid* grid, double* edges_host);
mf_status mf_grid_set(mf_grid* grid, const double* edges_host);
/* Forget the recorded iterations (the combination starts again). */
mf_status mf_grid_reset(mf_grid* grid);
/* The recorded iterations (checkpoint / resume of the combination): with
 * I_k and var_k NULL, *count receives the number recorded; otherwise the
 * first *count estimates I_k and variances sigma_k^2 are copied to the host
 * arrays (*count must be >= the number recorded).  mf_grid_set_history
 * replaces the record with `count` iterations (every var_k > 0).  Together
 * with mf_grid_get/set and the counter-based random numbers, a restored grid
 * continues like the original: the same events and per-event weights; the
 * iteration sums differ only in summation order (~1e-16 relative). */
mf_status mf_grid_history(const mf_grid* grid, int* count, double* I_k, double* var_k);
mf_status mf_grid_set_history(mf_grid* grid, int count, const double* I_k, const double* var_k);

/* The uniforms alone (arXiv:2211.14056 Sec. 1: the tensorised Monte Carlo
 * draws a tensor of random numbers per iteration; Philox4x32-10, Salmon et
 * al., SC'11): y[j][e] in [0, 1) for dimension j < ndim of global event
 * first_event + e, e < n, the stream every sampling kernel of this library
 * draws from (key (seed_lo, seed_hi ^ iter), counter (event_lo, event_hi,
 * j/2, 0), dims 2k and 2k+1 from words (0,1) and (2,3), 53-bit mantissas).
 *   y  device [ndim][n] FP64, caller-owned (output); 1 <= ndim <= 10.
 * Asynchronous on `stream`.  MF_ERR_ARG: negative n or first_event, ndim out
 * of range, y NULL with n > 0. */
mf_status mf_uniforms(uint64_t seed, int iter, int64_t first_event, int64_t n, int ndim, double* y, void* stream);

/* Per-event kinematics of global events 0..n-1 of iteration `iter`:
 * Philox4x32-10 uniforms, Vegas map, luminosity map, RAMBO on diet, massive
 * rescaling, cuts.  Outputs (device, each may be NULL):
 *   momenta   [n_ext][4][n] FP64 (see conventions);
 *   weight_ps [n] FP64: the event weight without |M|^2 (0 if cut or Newton miss);
 *   bins      [ndim][n] uint8 Vegas bin of each dimension. */
mf_status mf_sample(mf_process* proc, const mf_grid* grid, uint64_t seed, int iter, int64_t n, double* momenta,
                    double* weight_ps, uint8_t* bins, void* stream);

/* Spin/colour averaged |M|^2 of n events (Sec. 2's device operator):
 *   momenta [n_ext][4][n] FP64 device, me2 [n] FP64 device. */
mf_status mf_matrix_element(mf_process* proc, int64_t n, const double* momenta, double* me2, void* stream);

/* Helicity sampling (the paper sums the helicities inside its operator,
 * Sec. 2; MadEvent and MadFlow can instead draw one configuration per event).
 * A configuration h of g g -> t t~ + gluons fixes the helicities of the NG
 * gluons and of the antitop: bit g (g < NG, the gluons in MadGraph order, the
 * two incoming first) set means gluon g has helicity +1, bit NG set means the
 * antitop has helicity +1; the top's two helicities are always summed.  For
 * the two-quark-line processes (MF_PROC_UUX_TTXGG and MF_PROC_UXU_TTXGG ..
 * MF_PROC_GUX_TTXGUX) h has 5 bits, those of the u u~ -> t t~ g g
 * amplitude's slots that the channel fills, each the helicity of the
 * physical particle there: bit 0 the incoming quark of the light line (the
 * incoming antiquark for u~ g and g u~, whose amplitude is the charge
 * conjugate), bit 1 the other light fermion (the incoming antiquark, or the
 * outgoing (anti)quark of the q g channels), bit 2 the heavy fermion in the
 * antitop slot (the antitop; the top for u~ g and g u~), bits 3 and 4 the
 * gluons (the incoming one first in the q g channels); the other heavy
 * fermion's two helicities are summed.
 *
 * mf_matrix_element_hel: me2[e] = (1 / average) (|M(h_e, t-)|^2 + |M(h_e, t+)|^2)
 * of event e at configuration hel[e] (int32 device array [n], only the low
 * NG + 1 bits are read), momenta as mf_matrix_element; summed over the
 * 2^(NG+1) (32) configurations it is mf_matrix_element's value.  Covers the
 * gluon-initiated and the two-quark-line processes in MF_FP64 and MF_FP32
 * (else MF_ERR_UNSUPPORTED).
 *
 * mf_set_helicity_sampling(proc, on), on = 1: from then on the process's
 * iterations (mf_vegas_accumulate, mf_vegas_iterate, mf_unweight) estimate
 * |M|^2 of each event by mf_matrix_element_hel / p_h at a configuration h
 * drawn from the grid's helicity table: with w0 word 0 of Philox4x32-10 under
 * the Vegas key (seed & 0xffffffff, (seed >> 32) ^ iter) and counter
 * (event & 0xffffffff, event >> 32, 1, 1), h = max{h : T_h <= w0} for the
 * table's thresholds 0 = T_0 <= ... <= T_H = 2^32 (H = 2^(NG+1)), and p_h =
 * (T_{h+1} - T_h) / 2^32.  A new grid's table is uniform (T_h = h 2^32 / H:
 * h is the top log2(H) bits of w0, the weight H |M_h|^2; H = 2^(NG+1), or 32
 * for the two-quark-line processes).  on = 2 also
 * sums, per configuration, the squared weights of the events that drew it
 * (appended to the totals of mf_grid_totals) so that mf_vegas_finish with
 * refine bit 2 refines the table: q_h = sqrt(p_h S_h), p'_h = 0.9 q_h / sum(q)
 * + 0.1 / H (every sum in configuration order), T'_h = floor(2^32 (p'_0 + ...
 * + p'_{h-1})); a table whose S are all zero stays.  The estimate is unbiased
 * for any table with every p_h > 0; its variance is larger than the sum's,
 * its cost per event smaller.  0 restores the sum.  The launch shape
 * (mf_set_launch_shape) applies to the summed kernel only.  Not covered while
 * it is on: mf_vegas_accumulate_static, mf_grad, mixed plans
 * (MF_ERR_UNSUPPORTED).  Errors: MF_ERR_ARG (on not 0, 1 or 2),
 * MF_ERR_UNSUPPORTED (e+ e- -> mu+ mu-, or MF_FP32_TC). */
mf_status mf_matrix_element_hel(mf_process* proc, int64_t n, const double* momenta, const int32_t* hel, double* me2,
                                void* stream);
mf_status mf_set_helicity_sampling(mf_process* proc, int on);

/* The grid's helicity table as probabilities p[0..n-1] (host, n = 2^(NG+1)):
 * mf_grid_helicity reads them (p_h = (T_{h+1} - T_h) / 2^32, exact);
 * mf_grid_set_helicity sets the thresholds T_h = floor(2^32 (p_0 + ... +
 * p_{h-1})) (partial sums added in order), which mf_grid_helicity then
 * returns exactly.  Synchronous.  Errors: MF_ERR_ARG (wrong n, a p_h that is
 * not finite and > 0 or that leaves its configuration no threshold step,
 * sum not 1 within 1e-9), MF_ERR_UNSUPPORTED (the process has no helicity
 * table: e+ e- -> mu+ mu- has none). */
mf_status mf_grid_helicity(const mf_grid* grid, double* prob, int n);
mf_status mf_grid_set_helicity(mf_grid* grid, const double* prob, int n);

/* One Vegas iteration over global events 0..n-1 (chunks of 2^20 events: a
 * sampling kernel writes per-event records and the list of events passing the
 * cuts, the |M|^2 kernel reads them and accumulates), a deterministic reduction of the per-CTA
 * sums, and the refinements that refine asks for: bit 1 the Vegas edges,
 * bit 2 the helicity table (processes with mf_set_helicity_sampling(proc, 2);
 * other values are MF_ERR_ARG).  The iteration is recorded
 * on the grid and *out (host) receives it and the running combination.
 * weights (device [n] FP64, may be NULL) receives every event weight.
 * Synchronises the stream.  Returns MF_WARN_NEWTON if any event missed the
 * Newton tolerance. */
mf_status mf_vegas_iterate(mf_process* proc, mf_grid* grid, uint64_t seed, int iter, int64_t n, int refine,
                           mf_result* out, double* weights, void* stream);

/* The same iteration in two halves, for event sharding across devices
 * (the Philox counter is the global event index, so a shard is events
 * first_event .. first_event+n-1 and the result does not depend on the split):
 *   mf_vegas_accumulate runs the iteration's kernels on the shard and reduces its
 *     per-CTA partial sums into the grid's totals buffer (asynchronous);
 *   mf_grid_totals exposes that device buffer, double[count] laid out as
 *     [0] sum w, [1] sum w^2, [2 + j*nbins + b] sum w^2 in bin b of dim j,
 *     then events passing cuts and Newton misses, then (adaptive helicity
 *     sampling) the sums of squared weights of the 2^(NG+1) configurations,
 *     so that the caller can all-reduce it (sum) over shards; the library owns it;
 *   mf_vegas_finish turns the (summed) totals of n_total events into the
 *     estimate, refines as refine asks, records the iteration and fills
 *     *out like mf_vegas_iterate (synchronises the stream). */
mf_status mf_vegas_accumulate(mf_process* proc, mf_grid* grid, uint64_t seed, int iter, int64_t first_event,
                              int64_t n, double* weights, void* stream);
mf_status mf_grid_totals(mf_grid* grid, double** totals_device, int* count);
mf_status mf_vegas_finish(mf_process* proc, mf_grid* grid, int64_t n_total, int refine, mf_result* out, void* stream);

/* Allocation-free mf_vegas_accumulate (the paper has no counterpart: it is an
 * interface for host programs that forbid the libraries they load from
 * allocating device memory, e.g. a framework that hands out all device memory
 * from its own arena, or a process whose memory budget is already spent).
 * Same computation as mf_vegas_accumulate, but the caller passes every buffer:
 *   edges   device [ndim][nbins+1] FP64 Vegas edges (input; 2 <= nbins <= 64);
 *   totals  device double[2 + ndim*nbins + 2] (output, layout of mf_grid_totals);
 *   weights device [n] FP64 or NULL (output).
 * The per-CTA scratch lives in a fixed 2 MiB array inside the library's device
 * image, reserved on every device that loads the library until the process
 * exits; the launch uses as many persistent CTAs as that array holds (the
 * result does not depend on the CTA count), and a set-up whose single CTA
 * needs more than the array returns MF_ERR_ARG.  MF_ERR_UNSUPPORTED: the
 * fused kernel does not fit on an SM.  The first call on a device looks up
 * that array's device address and caches it for the process (make that call
 * before any stream capture); the cached address does not survive
 * cudaDeviceReset, after which this entry point must not be called again in
 * the process.  The call allocates nothing.  All calls on a device share the one
 * array: calls that overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  Each call overwrites every scratch
 * word it reads, so nothing needs clearing between calls. */
mf_status mf_vegas_accumulate_static(mf_process* proc, const double* edges, int nbins, uint64_t seed, int iter,
                                     int64_t first_event, int64_t n, double* totals, double* weights, void* stream);

/* Unweighted events by hit-or-miss (the event-generation step that follows
 * the weighted integration of arXiv:2211.14056 Sec. 1; the paper states no
 * algorithm, this is the practice of MadEvent/MadFlow): the events
 * first_event .. first_event + n - 1 of iteration `iter` are evaluated on the
 * grid's current edges exactly as by mf_vegas_iterate (same weights w; the
 * grid records nothing), and event e is kept if r_e w_max < w_e, with r_e the
 * uniform of a second Philox stream (same key, counter (e_lo, e_hi, 0, 1),
 * words (0, 1)).  A kept event carries weight max(1, w_e / w_max) (> 1 for an
 * overweight event), so that w_max * (sum of kept weights) / n estimates the
 * integral without bias.  Outputs (device, caller-owned, `capacity` entries
 * each): momenta [n_ext][4][capacity] FP64 (the event's momenta in the layout
 * of the conventions, from the kinematics the weight was computed with),
 * weight [capacity] FP64, event [capacity] int64 (global event index).  The
 * kept events are written in an unspecified order (their set is fixed).
 * *n_kept, *n_over (host): events kept, of which overweight.  More kept
 * events than `capacity`: only `capacity` are written and the call returns
 * MF_WARN_CAPACITY.  MF_ERR_ARG: w_max not finite and > 0, bad sizes.
 * Synchronises the stream. */
mf_status mf_unweight(mf_process* proc, mf_grid* grid, uint64_t seed, int iter, int64_t first_event, int64_t n,
                      double w_max, int64_t capacity, double* momenta, double* weight, int64_t* event,
                      int64_t* n_kept, int64_t* n_over, void* stream);

/* Derivatives of one iteration's estimate (arXiv:2211.14056 Sec. 2: the
 * device operator is differentiable in principle; the paper leaves its
 * derivative for later).  Over global events 0..n-1 of iteration `iter` on the
 * grid's current edges (the same events and weights as mf_vegas_iterate):
 *   *sigma          host: I = (1/n) sum w, in pb;
 *   dsigma          host double[3]: dI/dg_s, dI/dm_t, dI/dGamma_t at the
 *                   process's parameters (m_t moves the external top masses,
 *                   the phase-space threshold and the propagators together);
 *   dw_dtheta       device [3][n] FP64 or NULL: per-event dw/dg_s, dw/dm_t,
 *                   dw/dGamma_t;
 *   dw_dy           device [ndim][n] FP64 or NULL: per-event dw/dy_j, the
 *                   derivative with respect to the Vegas uniform of
 *                   dimension j inside its bin.
 * Reverse mode: per chunk of events, the sampler runs with two tangents (m_t
 * and y_0) and writes per-event records; the adjoint kernel recomputes every
 * wavefunction, current and amplitude of |M|^2 and sweeps back once to
 * d|M|^2/d(momenta, m_t, Gamma_t), which it contracts with the records'
 * tangents and keeps per event; with dw_dy, further sampler-only passes
 * carry two uniforms each and reuse the stored adjoint.  dI/dg_s is exact:
 * |M|^2 is proportional to g_s^(2 n_gluons).  Bins, cuts and the Newton
 * decision are piecewise constant and give no derivative, so dI/dtheta is
 * the derivative of the estimator at fixed uniforms, not of the integral
 * across a moving cut boundary.  Arithmetic in the process's precision
 * (FP32 kinematics and amplitudes with MF_FP32, the weight in FP64).  Uses
 * the grid's scratch; synchronises the stream. */
mf_status mf_grad(mf_process* proc, const mf_grid* grid, uint64_t seed, int iter, int64_t n, double* sigma,
                  double* dsigma, double* dw_dtheta, double* dw_dy, void* stream);

/* The same derivatives in forward mode (the cross-check of mf_grad): every
 * pass recomputes the kinematics and |M|^2 with dual numbers carrying two
 * tangent directions; pass 0 carries m_t and Gamma_t, each further pass (only
 * with dw_dy) two uniforms.  Same arguments, outputs and errors as mf_grad. */
mf_status mf_grad_forward(mf_process* proc, const mf_grid* grid, uint64_t seed, int iter, int64_t n, double* sigma,
                          double* dsigma, double* dw_dtheta, double* dw_dy, void* stream);

/* Measurement utility: when enabled, mf_vegas_accumulate records CUDA events
 * around its per-chunk kernels (the iteration runs in chunks of 2^20 events:
 * a sampling kernel writes per-event records, the |M|^2 kernel reads them);
 * mf_grid_profile_read waits for the last call's events and returns the
 * summed device time of the sampling kernels and of the |M|^2-and-accumulate
 * kernels, and the number of chunks (the per-launch time of the |M|^2 kernel
 * is me_ms / chunks). */
mf_status mf_grid_profile(mf_grid* grid, int enable);
mf_status mf_grid_profile_read(mf_grid* grid, double* sample_ms, double* me_ms, int* chunks);

/* Measurement utility: sustained FMA-pipe throughput of the current device
 * (MF_FP32 or MF_FP64) in TFLOP/s from independent FMA chains on every SM,
 * the denominator of the amplitude kernel's roofline.  Synchronises the device. */
mf_status mf_fma_throughput(int precision, double* tflops);

/* Mixed launch: up to 8 processes integrated together, each with its own
 * grid and event count (arXiv:2211.14056 Sec. 3, Fig. 3: how the work is
 * spread over blocks and threads sets the run time).  One sampling launch
 * for every process, one persistent |M|^2 launch whose warps take tiles of
 * events from a single work queue ordered by cost (most gluons first), then
 * the per-process reduction and refinement.  The processes must share a
 * precision; grids belong to their processes.
 *   mf_mixed_create   reserves per-event records for n[k] events on each grid
 *                     (a configuration call; device memory grows once);
 *   mf_mixed_run      one iteration, out[k] receives process k's result like
 *                     mf_vegas_iterate (synchronises the stream);
 *   mf_mixed_set_launch  CTAs per SM of the |M|^2 launch (0 = occupancy) and
 *                     events per work item; tile = 0 selects the per-process
 *                     form instead: no shared queue, every process runs its own
 *                     specialised |M|^2 kernel (most gluons first) at its own
 *                     occupancy, inside the same iteration (and graph);
 *   mf_mixed_use_graph  capture the whole iteration as a CUDA graph on the
 *                     next run (per stream and refine flag) and replay it with
 *                     a new seed/iteration (copied from pinned host memory by
 *                     a node of the graph); the legacy default stream (NULL)
 *                     cannot be captured, so there the iteration runs uncaptured;
 *   mf_mixed_autotune times each candidate (ctas_per_sm, tile), tile = 0
 *                     being the per-process form, on one unrefined iteration
 *                     (results not recorded), writes the times (ms) and the
 *                     index of the fastest, and keeps it.
 * When the shared-queue kernel cannot fit on an SM (its shared memory holds
 * every process's Vegas sums beside the warps' g g -> t t~ g g stores: e.g.
 * seven FP64 processes), the plan runs the per-process form only: tile > 0
 * in mf_mixed_set_launch or in an autotune candidate is MF_ERR_UNSUPPORTED. */
typedef struct mf_mixed mf_mixed;
mf_status mf_mixed_create(mf_process* const* procs, mf_grid* const* grids, const int64_t* n, int nproc,
                          mf_mixed** out);
mf_status mf_mixed_destroy(mf_mixed* plan);
mf_status mf_mixed_run(mf_mixed* plan, uint64_t seed, int iter, int refine, mf_result* out, void* stream);
mf_status mf_mixed_set_launch(mf_mixed* plan, int ctas_per_sm, int tile);
mf_status mf_mixed_use_graph(mf_mixed* plan, int enable);
mf_status mf_mixed_autotune(mf_mixed* plan, uint64_t seed, int ncand, const int* cand_ctas, const int* cand_tile,
                            double* ms, int* best, void* stream);

/* Message of the last failing call on the calling thread ("" if none). */
const char* mf_last_error(void);

/* Number of device kernels the library launched since load (all threads). */
int64_t mf_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* MADFLOW_GB300_H */
