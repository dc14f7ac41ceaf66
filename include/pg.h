/*
 * pg.h -- C ABI of the GB300 pairwise-force library.
 *
 * The library evaluates the i-particle x j-particle force loop of
 * Phantom-GRAPE (Tanikawa, Yoshikawa, Nitadori & Okamoto 2012,
 * arXiv:1203.4037) on one NVIDIA GB300 GPU, in two forms:
 *
 *   PG_NEWTON  Eq. (1) with G = 1 and Plummer softening eps:
 *              a_i = sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2),
 *              phi_i = -sum_j m_j / (|x_j - x_i|^2 + eps^2)^(1/2)
 *              (the potential's sign is the one of the Newton force loop of
 *              Section 3.3, which subtracts m/r from the potential);
 *   PG_TABLE   Eq. (2): a_i = sum_j m_j g(|x_j - x_i|) (x_j - x_i), with
 *              g = f(r)/r read from the bit-pattern table of Section 3.4
 *              (E exponent bits, F fraction bits, linear interpolation in
 *              s = r^2 (s_max - 2) / r_cut^2 + 2) and g = 0 for r >= r_cut.
 *              No potential is computed in this mode (as in the paper).
 *
 * The call sequence follows the GRAPE-5 style API of Section 3.6
 * (g5_open / g5_set_eps_to_all / g5_set_n / g5_set_xmj /
 * g5_calculate_force_on_x / g5_close) plus the paper's table setter.
 *
 * Conventions for every entry point:
 *   - positions are row-major double[n][3], masses double[n] (FP64);
 *   - "host" pointers are ordinary CPU memory the caller owns; the library
 *     copies what it needs before returning (set_*) or writes into them
 *     (get_*); "dev" pointers are CUDA device memory on the context's device,
 *     borrowed only for the duration of the work the call enqueues on the
 *     context's stream;
 *   - calls are asynchronous on the context's stream unless stated; the
 *     library never synchronises the device except in pg_get_force,
 *     pg_get_table, pg_sync, pg_tune and pg_selftest_wait, and in the
 *     setters that copy from host arrays through pageable memory
 *     (pg_set_table, pg_set_table_values,
 *     pg_set_table_pot, pg_set_table_pot_values, pg_set_eps_i), which wait
 *     for the context's stream before they return;
 *   - a context is not thread-safe; use one per host thread;
 *   - every function returns PG_OK (0) or a negative status; it never aborts
 *     the process and never traps the GPU. pg_last_error() describes the last
 *     failure. A device-side wait that runs out of time (PG_ETIMEOUT) is
 *     reported by the next synchronising call.
 */
#ifndef PG_H
#define PG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pg_ctx pg_ctx;

/* status codes */
#define PG_OK 0
#define PG_EINVAL (-1)    /* bad argument (negative size, E+F out of range, r_cut <= 0, ...) */
#define PG_ESTATE (-2)    /* call out of order (run before j/i/table were set, ...) */
#define PG_ENOMEM (-3)    /* device or pinned host allocation failed */
#define PG_ECUDA (-4)     /* a CUDA runtime call failed */
#define PG_ETIMEOUT (-5)  /* a device-side bounded wait gave up */

/* force modes (pg_set_mode) */
#define PG_NEWTON 0
#define PG_TABLE 1

/* all-pairs paths (pg_set_allpairs_path) */
#define PG_PATH_AUTO 0    /* narrow for ni <= 4096 against nj >= 64 ni, else tiled */
#define PG_PATH_TILED 1   /* i tiles of 256 to 1024 particles, j split across CTAs */
#define PG_PATH_NARROW 2  /* few i against many j: (i chunk, j chunk) items */

/* how the all-pairs paths form pair differences (pg_set_differencing) */
#define PG_DIFF_AUTO 0    /* double-float where i-tiles are not compact (the default) */
#define PG_DIFF_SINGLE 1  /* one FP32 offset per particle from an FP64 tile centre */
#define PG_DIFF_DOUBLE 2  /* double-float on every all-pairs run */

/* long-range split of the particle-mesh part (pg_set_pm) */
#define PG_SPLIT_GAUSS 0  /* D(k) = exp(-k^2 r_s^2): the erf split of the Gaussian-split PP shape */
#define PG_SPLIT_S2 1     /* D(k) = S(k a)^2: Hockney and Eastwood's S2 clouds of diameter a */

/* Open a context on CUDA device `device` (g5_open, Section 3.6; no rsqrt
 * bias calibration: the GPU's rsqrt has a documented error bound instead).
 * *out receives the handle; destroy it with pg_destroy. The context starts
 * on an internal non-blocking stream of its own (pg_set_stream changes it). */
int pg_create(pg_ctx **out, int device);

/* Release every resource of the context (g5_close). NULL is ignored. */
void pg_destroy(pg_ctx *ctx);

/* Enqueue all later work on `cuda_stream` (a cudaStream_t owned by the
 * caller, e.g. the current PyTorch stream); NULL is the CUDA legacy default
 * stream. Work already enqueued is ordered before later work. */
int pg_set_stream(pg_ctx *ctx, void *cuda_stream);

/* Plummer softening length used by PG_NEWTON (g5_set_eps_to_all,
 * Section 3.6): eps >= 0, one value for all particles. With eps = 0 a pair
 * at zero distance contributes nothing. */
int pg_set_eps(pg_ctx *ctx, double eps);

/* Softening per i-particle: the i-particle structure of Section 3.1 carries
 * eps^2 per particle, and the Newton kernel of Section 3.3 adds the
 * i-particle's eps^2 to |d|^2. eps: host double[n], finite and >= 0 (copied;
 * PG_EINVAL otherwise). n must equal the i count of pg_set_i when pg_run runs
 * (PG_ESTATE otherwise). In self mode the left-out own pair is the one with
 * the i-particle's eps. NULL or n = 0 returns to the global eps of
 * pg_set_eps. PG_NEWTON only (pg_run returns PG_ESTATE in PG_TABLE mode); the
 * backward pass refuses it (PG_ESTATE). Waits for the context's stream. */
int pg_set_eps_i(pg_ctx *ctx, const double *eps, long long n);

/* The same from a device array (double[n]; a negative value acts as its
 * absolute value), copied in stream order. */
int pg_set_eps_i_dev(pg_ctx *ctx, const double *eps, long long n);

/* Select PG_NEWTON (default) or PG_TABLE. */
int pg_set_mode(pg_ctx *ctx, int mode);

/* Build the force table from a host callback (the paper's non-GRAPE-5
 * table setter, Section 3.6; construction of Section 3.4.1):
 *   g(r, user) returns f(r)/r for 0 <= r <= r_cut (finite at r = 0);
 *   knot k = 2^F bE + bF sits at s_k = 2^(bE+1) (1 + bF/2^F), i.e. at
 *   r_k = r_cut sqrt((s_k - 2) / (s_max - 2)), s_max = 2^(2^E) (2 - 2^-F);
 *   v_k = (float) g(r_k) for every knot, the last knot being r_cut itself;
 *   stored G0_k = v_k and G1_k = (v_{k+1} - v_k) / (s_{k+1} - s_k) (rounded
 *   once to FP32) for k < 2^(E+F) - 1; the last entry is G0 = G1 = 0, so the
 *   force is zero at and beyond r_cut.
 * Requires r_cut > 0, E >= 0, F >= 0, 1 <= E + F <= 13, E <= 7, F <= 20.
 * The callback runs on the calling thread, 2^(E+F) times, before return. */
int pg_set_table(pg_ctx *ctx, double (*g)(double r, void *user), void *user, double r_cut,
                 int E, int F);

/* The same table from knot values v[0 .. n-1] (host, FP32), n = 2^(E+F);
 * v[n-1] is g at r_cut approached from below. */
int pg_set_table_values(pg_ctx *ctx, const float *v, long long n, double r_cut, int E, int F);

/* The same from device knot values (FP32, n = 2^(E+F)); the table is
 * derived on the GPU. Used for trainable tables. */
int pg_set_table_values_dev(pg_ctx *ctx, const float *v, long long n, double r_cut, int E,
                            int F);

/* Copy the stored table (G0, G1: FP32 host arrays of n = 2^(E+F)). Syncs. */
int pg_get_table(pg_ctx *ctx, float *G0, float *G1, long long n);

/* Tree front end: the tree usage of Section 5.1 (a Barnes-Hut tree, vacuum
 * boundary, monopole moments; i-particles in groups that traverse the tree
 * once and share one interaction list). With theta >= 0 every later pg_run
 * computes the forces and potentials of all particles this way: the tree is
 * built over the j-particles on the GPU, each group of at most ncrit
 * particles (a tree node) collects its list of particles and node
 * pseudo-particles, and the batched-group kernel evaluates the lists; a
 * particle's own pair is left out. Construction and opening rule:
 *   - nodes are the runs of equal 3L-bit prefix of a 30-bit Morton key
 *     (10 bits per axis over the bounding cube), levels 0 .. 10;
 *   - a node holding none of the group's particles is accepted if
 *     side^2 < theta^2 d^2, d from its centre of mass to the group's box,
 *     and enters the list as its pseudo-particles (see
 *     pg_set_tree_quadrupole);
 *   - otherwise a leaf (at most nleaf particles, or level 10) gives its
 *     particles and other nodes are opened.
 * theta = 0 reproduces the direct sum. Needs PG_NEWTON, the self mode with
 * ni == nj, no groups, no periodic box and the global eps (PG_ESTATE
 * otherwise). A tree run synchronises once, at its end, to read its
 * counts back: the call sizes every buffer from the previous call's counts
 * (with an eighth and 256 more room); when a count outgrows its room, or on
 * the first call for a particle count, it reads each count back before the
 * stage that needs it instead (pg_get_tree_stats tells which ran). It is
 * not captured in a graph. theta < 0 turns it off.
 * A run returns PG_EINVAL when the particles plus pseudo-particles reach
 * 2^27 (the list index width) or the lists reach 2^32 entries.
 * PG_EINVAL for a theta that is not finite, ncrit outside 1 .. 2^20 or
 * nleaf < 1. */
int pg_set_tree(pg_ctx *ctx, double theta, int ncrit, int nleaf);

/* The pseudo-particles of an accepted tree node (the paper's monopole and
 * quadrupole tree runs, Section 5.1). on = 0 (the default): one, the node's
 * mass at its centre of mass c. on != 0: the pseudo-particle multipole
 * method of Kawai and Makino at quadrupole order, three of mass M / 3 at
 * c + a e1 and c - a/2 e1 +- (sqrt 3 / 2) b e2, where e1, e2 are the unit
 * principal axes of the node's second moment T = sum m (x - c)(x - c)^T
 * with its two largest eigenvalues l1 >= l2 (l3 the smallest; e1's
 * largest component positive), a = sqrt(2 (l1 - l3) / M) and
 * b = sqrt(2 (l2 - l3) / M): they carry the node's mass, a zero dipole and
 * the trace-free part of T. Moments in FP64; the opening test is the same.
 * Takes effect at the next run. */
int pg_set_tree_quadrupole(pg_ctx *ctx, int on);

/* The last tree run's structure, for inspection: sizes[6] = {n, nodes,
 * groups, list entries, work items, P pseudo-particles per node}; then
 * (each may be NULL) perm[n] (key order -> input index), the groups' first
 * particle and size in key order [groups], j_off[groups + 1] and
 * jlist[list entries] (k < n: particle k in key order; n + P t + q:
 * pseudo-particle q of node t, nodes numbered level by level; a list runs
 * breadth first, level by level and in key order within a level). Syncs. */
int pg_get_tree(pg_ctx *ctx, long long *sizes, long long *perm, long long *g_i0,
                long long *g_ni, long long *j_off, long long *jlist);

/* How the tree walk runs (both make the same lists).
 * PG_TREE_WALK_AUTO (the default): one warp walks one group breadth first,
 * holding the nodes the group opened at the previous level (at most 512,
 * PG_TREE_WALK_QUEUE) in shared memory; a group that opens more on one
 * level (a small theta) makes the call use the level walk.
 * PG_TREE_WALK_LEVEL: the level walk always: all groups level by level,
 * one thread per (group, node) visit, with the next level's size read back
 * between levels. PG_EINVAL for another mode. */
#define PG_TREE_WALK_AUTO 0
#define PG_TREE_WALK_LEVEL 1
#define PG_TREE_WALK_QUEUE 512
int pg_set_tree_walk(pg_ctx *ctx, int mode);

/* The last tree run's execution: out[0] the walk that made the lists
 * (1 group walk, 2 level walk), out[1] 1 if the run read each count back
 * before the stage that needs it, 0 if it ran from the previous call's
 * room, out[2] the most nodes one group opened on one level (group walk;
 * above PG_TREE_WALK_QUEUE when it gave up), out[3] the host read-backs of
 * the call (counting the run from room that came out too small, if any).
 * Writes min(nout, 4) values. */
int pg_get_tree_stats(pg_ctx *ctx, long long *out, int nout);

/* The particle-mesh (PM) long-range force of the PPPM and TreePM methods
 * whose short-range part the arbitrary-shape force loop evaluates (Section
 * 4.2: PP with f(r) = R(r, eps) - R(r, r_cut) plus PM with R(r, r_cut) make
 * the full softened force). In the periodic cube of pg_set_periodic (side
 * L), on an ngrid^3 mesh: TSC mass assignment, FFT, the Green's function
 * -4 pi D(k) / k^2 with the split factor D (split = PG_SPLIT_GAUSS, scale
 * = r_s; or PG_SPLIT_S2, scale = the S2 diameter a) divided twice by the
 * TSC window, the k = 0 mode and the Nyquist planes dropped, spectral
 * gradient, TSC interpolation. FP32 mesh and FFTs (see pg_set_pm_fft),
 * FP64 in and out.
 * Once set, a pg_run in the periodic (cell-list) mode returns PP + PM:
 * the mesh forces at the i-particles from the j-particles are added to the
 * PP forces (and the mesh potential, which includes each particle's own
 * smoothed self-potential, to the PP potential). ngrid <= 0 turns it off.
 * PG_EINVAL for an odd ngrid or one outside 8 .. 1024, another split, or a
 * scale that is not finite and positive. */
int pg_set_pm(pg_ctx *ctx, int ngrid, int split, double scale);

/* The FFTs of the PM solve. PG_FFT_AUTO (the default): hand-written FFTs
 * for a power-of-two mesh from 8 to 512 (a radix-4 Stockham FFT per line in
 * shared memory; five passes over the mesh with the Green's function and
 * the spectral gradient applied inside them), cuFFT for other sizes.
 * PG_FFT_LIBRARY: cuFFT for every size (one real-to-complex transform, the
 * Green's function, a batch of four complex-to-real transforms). Both
 * compute the same fields up to FP32 rounding. pg_get_pm_fft writes to
 * *kind which the last PM solve used: 1 hand-written, 2 cuFFT, 0 none yet.
 * PG_EINVAL for another mode or a NULL kind. */
#define PG_FFT_AUTO 0
#define PG_FFT_LIBRARY 1
int pg_set_pm_fft(pg_ctx *ctx, int mode);
int pg_get_pm_fft(pg_ctx *ctx, int *kind);

/* The PM long-range acceleration a[3 n] and potential phi[n] (may be NULL)
 * of n particles x[3 n], m[n] on each other, alone (positions are wrapped
 * into the box). Host arrays; synchronises. PG_ESTATE without pg_set_pm or
 * pg_set_periodic. */
int pg_pm_forces(pg_ctx *ctx, const double *x, const double *m, long long n, double *a, double *phi);

/* The same on device arrays (FP64), enqueued on the context's stream. */
int pg_pm_forces_dev(pg_ctx *ctx, const double *x, const double *m, long long n, double *a,
                     double *phi);

/* The mesh force in two steps, for particles split across ranks (each rank
 * deposits its own particles, the ranks sum the meshes, and each solves for
 * its own). pg_pm_deposit_dev writes the density of n particles (device
 * FP64 x[3 n], m[n]) into rho: ngrid^3 FP32 values in device memory the
 * caller owns, row-major with z fastest, mass per cell volume.
 * pg_pm_solve_dev takes such a mesh (summed over ranks; it is not changed)
 * and writes the acceleration a[3 n] and potential phi[n] (may be NULL) at
 * n positions x[3 n]. Deposit then solve on the same particles equals
 * pg_pm_forces_dev. Enqueued on the context's stream; PG_ESTATE without
 * pg_set_pm or pg_set_periodic. */
int pg_pm_deposit_dev(pg_ctx *ctx, const double *x, const double *m, long long n, float *rho);
int pg_pm_solve_dev(pg_ctx *ctx, const float *rho, const double *x, long long n, double *a, double *phi);

/* The last tree run's pseudo-particles: rec[4 P nodes] = x, y, z, m (FP64)
 * of pseudo-particle q of node t at 4 (P t + q), host memory the caller
 * owns. Syncs. */
int pg_get_tree_pseudo(pg_ctx *ctx, double *rec);

/* Potential in PG_TABLE mode, an extension: the tabulated kernel of Section
 * 3.4.2 stores accelerations only. psi(r, user) is tabulated on the force
 * table's knots (same r_cut, E, F) and built the same way, including the
 * cutoff reading: psi~ = 0 at and beyond r_cut, and the last interior bin
 * runs to psi(r_cut) from below. Then phi_i = sum_j m_j psi~(s_ij); in self
 * mode without the own pair. Needs the force table first (PG_ESTATE);
 * p = NULL drops the potential (phi is zero again). A later force table with
 * the same r_cut, E, F keeps the potential; another geometry drops it. The
 * table in shared memory doubles (16 B per knot). Waits for the stream. */
int pg_set_table_pot(pg_ctx *ctx, double (*p)(double r, void *user), void *user);

/* The same from knot values v[0 .. n-1] (host FP32, n = 2^(E+F) of the force
 * table; v[n-1] is psi at r_cut from below). PG_EINVAL for another n or a
 * value that is not finite. */
int pg_set_table_pot_values(pg_ctx *ctx, const float *v, long long n);

/* Number of j-particles used by pg_run (g5_set_n). Without it, pg_run uses
 * the highest address written by pg_set_j / pg_set_j_dev. */
int pg_set_n(pg_ctx *ctx, long long nj);

/* Store j-particles adr .. adr+nj-1 (g5_set_xmj, Section 3.6): positions
 * x (host double[nj][3]) and masses m (host double[nj]). Copies: the
 * caller may reuse x and m when the call returns. Pageable memory is
 * copied into the context's page-locked staging buffer and sent from there
 * in stream order; page-locked (pinned) x and m are sent by DMA directly,
 * and the call then waits for that copy (and the stream's earlier work). */
int pg_set_j(pg_ctx *ctx, long long adr, long long nj, const double *x, const double *m);

/* Device twin of pg_set_j: x (device double[nj][3]), m (device double[nj]). */
int pg_set_j_dev(pg_ctx *ctx, long long adr, long long nj, const double *x, const double *m);

/* j-particles adr .. adr+nj-1 as packed records rec (device double[nj][4]:
 * x, y, z, m per particle, the library's own record layout), copied in
 * stream order with one device copy: for records that arrive packed, such
 * as a buffer all-gathered from every rank's particles each step. An
 * extension (the paper's API takes positions and masses apart). */
int pg_set_j_rec_dev(pg_ctx *ctx, long long adr, long long nj, const double *rec);

/* The i-particles of the next pg_run: x (host double[ni][3]). Copies, as
 * pg_set_j does (pinned x: by DMA, waited for). */
int pg_set_i(pg_ctx *ctx, long long ni, const double *x);

/* Device twin of pg_set_i. */
int pg_set_i_dev(pg_ctx *ctx, long long ni, const double *x);

/* on != 0: i-particle k is j-particle k (all-pairs use, the same arrays
 * given to set_j and set_i), and its own pair is left out of the sums, as
 * in the double-precision reference of Section 4.1. Requires ni <= nj and
 * bit-identical positions. on = 0 (default): every j counts. */
int pg_set_self(pg_ctx *ctx, int on);

/* Self mode with an offset, for an i-range that is part of the j-set:
 * i-particle k is j-particle lo + k (positions bit-identical), and its own
 * pair is left out of the sums as in pg_set_self. This is the self mode of
 * one rank of a run whose particles are split across ranks (each rank's
 * i-particles are its own slice of the all-gathered j records, which start
 * at lo). Requires lo + ni <= nj at pg_run (PG_ESTATE otherwise) and the
 * all-pairs paths (no groups, tree or periodic box: PG_ESTATE). lo = 0 is
 * pg_set_self(ctx, 1); pg_set_self(ctx, 0) turns the mode off. PG_EINVAL
 * for lo < 0. */
int pg_set_self_offset(pg_ctx *ctx, long long lo);

/* Batched tree-style lists (the usage of Section 5.1: each group of
 * i-particles shares one interaction list). Group g covers the i-particles
 * i_off[g] .. i_off[g+1]-1 (indices into the array of pg_set_i) and sums
 * exactly the j listed in jlist[j_off[g] .. j_off[g+1]-1] (indices into the
 * j array, 0 <= j < 2^27; repeats allowed; a listed self pair contributes
 * zero force and, in PG_NEWTON, -m/eps of potential). i_off and j_off are
 * int64[ngroups+1], non-decreasing, from 0; jlist is int32. Host arrays,
 * copied. While groups are set pg_run evaluates them instead of all pairs. */
int pg_set_groups(pg_ctx *ctx, long long ngroups, const long long *i_off, const long long *j_off,
                  const int *jlist);

/* Drop the groups: pg_run returns to all-pairs mode. */
int pg_clear_groups(pg_ctx *ctx);

/* Periodic cube of side box > 0 (PG_TABLE only): pg_run bins the
 * j-particles into a cell grid of side >= r_cut, sorts them by cell, and
 * sums over the 27 neighbour cells with minimum-image shifts (the PP
 * neighbour search of PPPM / TreePM codes). Requires r_cut <= box / 3 and the
 * self mode (the i-particles are the j-particles). box = 0 (default):
 * open boundaries. */
int pg_set_periodic(pg_ctx *ctx, double box);

/* Enqueue one force evaluation into the context's own output buffers. */
int pg_run(pg_ctx *ctx);

/* Copy the last results to the host: a (double[ni][3]) and phi (double[ni],
 * may be NULL; zeros in PG_TABLE mode). Synchronises; returns PG_ETIMEOUT
 * if a device wait gave up. ni must equal the count given to pg_set_i.
 * Page-locked (pinned) a and phi are written by DMA directly; others
 * through the context's page-locked staging buffer. */
int pg_get_force(pg_ctx *ctx, double *a, double *phi, long long ni);

/* Enqueue one force evaluation writing device outputs: a (device
 * double[ni][3]), phi (device double[ni] or NULL). */
int pg_run_dev(pg_ctx *ctx, double *a, double *phi);

/* Gradients of L = sum_i w_i . a_i for the all-pairs self mode
 * (i-particles = j-particles), recomputing the pair terms: w (device
 * double[n][3]) in; dx (device double[n][3]), dm (device double[n]) out; in
 * PG_TABLE mode also dv (device float[2^(E+F)]), the gradient with respect to
 * the knot values of the table (dv may be NULL). An extension: the paper has
 * no backward pass. */
int pg_backward_dev(pg_ctx *ctx, const double *w, double *dx, double *dm, float *dv);

/* The timeout path, checked on the device without a fault: one thread
 * waits, with the library's time-bounded wait and a limit of limit_ms
 * (0 < limit_ms <= 2000), on a barrier that nothing completes. The wait gives
 * up, and the call returns PG_ETIMEOUT as a timed-out run does; the status is
 * then cleared and the context stays usable. PG_OK would mean the wait did
 * not give up (a defect). Synchronises. */
int pg_selftest_wait(pg_ctx *ctx, double limit_ms);

/* Wait for the context's stream and report device-side status. */
int pg_sync(pg_ctx *ctx);

/* on != 0: pg_run / pg_run_dev capture their launch sequence in a CUDA graph
 * on first use and replay it while sizes, mode and buffers are unchanged. */
int pg_set_graph(pg_ctx *ctx, int on);

/* The autotuner: times the candidate launch shapes of the current workload
 * on the device (one warm-up run and three timed runs each) and keeps the
 * fastest in the context. Candidates: i per thread 2*np (np 1, 2, 4) on every
 * path; with it, on the tiled all-pairs path packed or scalar pair
 * arithmetic and CTAs per SM (the occupancy limit and one below); on the
 * batched kernel (groups, tree lists, cell list) CTAs per SM, and for the
 * caller's Newton groups (eps > 0, no per-i softening) also the kernel's
 * j-tile depth and threads per CTA (the shapes of pg_set_groups_tile); on
 * the narrow path the split of the j records into 1, 2 or 4 items per warp
 * of the launch. Synchronises. */
int pg_tune(pg_ctx *ctx);

/* Pair differences of the all-pairs paths (tiled and narrow). Positions are
 * FP64 (the inputs of Section 4.1); the pair loop runs in FP32. PG_DIFF_SINGLE
 * converts each particle once to an FP32 offset from its i-tile's FP64 centre
 * and differences the offsets: 13 FP32-pipe operations per Newton
 * interaction, with a difference error of about 2^-24 of the tile's extent,
 * small against |d| only when tiles are compact next to their close pairs.
 * PG_DIFF_DOUBLE also stages each offset's FP32 rounding residual and forms
 * d = (x~_j - x~_i) + (e_j - e_i): 3 more operations per component, an error
 * of a few 2^-24 of |d| itself whatever the tiles' extent. PG_DIFF_AUTO (the
 * default) takes single on PG_NEWTON tiled runs whose i-particles are
 * Morton-ordered (from 16384 on) and at least an eighth as many as the
 * j-particles, and double on every other tiled run (PG_TABLE included: the
 * shape's steep fall toward r_cut magnifies a difference's error) and on the
 * narrow path. pg_info's out[7] reports
 * what the last run used. Groups, tree lists and the cell list keep their
 * own forms. PG_EINVAL for another mode. */
int pg_set_differencing(pg_ctx *ctx, int mode);

/* The batched kernel's j-tile depth (j records staged in shared memory per
 * step) and threads per CTA for the caller's Newton groups (pg_set_groups;
 * eps > 0, no per-i softening): (512, 128) (the default, and the only shape
 * of every other batched run), (256, 128), (1024, 256) or (512, 256); (0, 0)
 * returns to the default. The group lists are cut into work items of at most
 * 2 np x threads i-particles. pg_info's out[8], out[9] report the shape of the
 * last batched launch. PG_EINVAL for a shape that is not compiled. */
int pg_set_groups_tile(pg_ctx *ctx, int tj, int nt);

/* Narrow all-pairs path: cut the j records into about items_per_warp work
 * items per warp of the launch (1 to 8; 0 = the default, one). pg_info's
 * out[6] reports the value a narrow run used. Returns PG_EINVAL outside
 * 0 to 8. */
int pg_set_split(pg_ctx *ctx, int items_per_warp);

/* Path of the all-pairs force loop (no groups, no periodic box); both give
 * the same sums up to FP32 rounding order. PG_PATH_TILED gives every CTA a
 * tile of i-particles in registers and a share of the j records, combining
 * the shares in FP64. PG_PATH_NARROW serves the individual time step regime
 * (Section 5: a step evaluates only the particles due for an update, often
 * tens to hundreds against all N): the i-set is cut into chunks and the j
 * records into chunks of equal length, every (i chunk, j chunk) pair is one
 * work item of the batched-group kernel (one warp per item when the i chunk
 * and the j chunk are small), and each i's FP64 partial sums are added in
 * j-chunk order. The path is chosen per call; pg_info's slots reports the
 * number of j chunks on the narrow path. Returns PG_EINVAL for another
 * value. */
int pg_set_allpairs_path(pg_ctx *ctx, int path);

/* Launch shape override: i per thread = 2*np (np in {1, 2, 4}; 0 = chosen
 * by problem size, the default),
 * CTAs per SM (0 = occupancy limit; for a periodic cell list whose small
 * cells go to the warp-mode kernel, one fewer, so that a block of that kernel
 * fits beside the CTA-mode kernel on every SM), packed = 1: pair arithmetic in packed
 * FP32x2 instructions, 0: scalar FP32 (same roundings), -1 = keep. */
int pg_set_shape(pg_ctx *ctx, int np, int ctas_per_sm, int packed);

/* on != 0: bracket the force kernel of every later run with CUDA events on
 * the context's stream, so that pg_kernel_time can report its duration. */
int pg_set_timing(pg_ctx *ctx, int on);

/* Duration in milliseconds of the force kernel of the last run (timing on;
 * waits for that kernel's end event). */
int pg_kernel_time(pg_ctx *ctx, double *ms);

/* Counters: out[0] pair evaluations enqueued by the last run, out[1] kernel
 * launches of the last run, out[2] i per thread, out[3] grid size of the
 * force kernel, out[4] partial slots per tile, out[5] 1 if the pair arithmetic
 * is packed FP32x2, out[6] items per warp of a narrow run (0 for other paths),
 * out[7] 1 if the pair differences were formed in double-float (FP32 offset
 * plus its FP32 residual: the narrow path, and tiled runs whose i-tiles are
 * not compact), 0 if from one FP32 offset per particle, out[8] and out[9]
 * the j-tile depth and threads per CTA of the batched kernel (0 when the run
 * did not use it).
 * Returns how many were written (at most 10). */
int pg_info(pg_ctx *ctx, long long *out, int n);

/* Measured ceilings on the current device for the roofline (a tool of this
 * library; the paper quotes only its CPU's peak): kind 0 scalar FP32 FMA,
 * 1 packed FP32x2 FMA (lane operations), 2 MUFU rsqrt, 3 the Newton pair
 * term with every operand in registers (interactions), 4 random 8-byte
 * gathers from a 4096-entry table in shared memory (lane gathers: the
 * tabulated force's lookup when a warp's pairs hit random bins), 5 the same
 * gathers from four interleaved copies of the table in shared memory (each
 * lane reads the copy of its lane index mod 4, which sits on its own quarter
 * of the banks; 1024-thread blocks, one per SM), 6 the same gathers through
 * the read-only global path from a table in device memory. Writes the rate per
 * SM per clock (at the device's maximum clock) and per second. Synchronises
 * the legacy default stream. */
int pg_microbench(int kind, double *per_sm_clock, double *per_second);

/* Largest particle count pg_newton_allpairs_noalloc accepts. */
#define PG_NOALLOC_MAX_N 16384

/* All-pairs Newton forces (as pg_set_self(ctx, 1) + pg_run_dev) for callers
 * that cannot allocate device memory at call time: a host application whose
 * memory pool has reserved the whole GPU (cudaMalloc would fail), or a
 * time-critical loop that must not stall on the device synchronisation that
 * cudaMalloc and cudaFree can cause. The paper has no counterpart; this is a
 * convenience of this library. The call uses no context and allocates nothing: its scratch is a
 * fixed array of about 3.6 MiB that every GPU loading the library holds
 * until the process exits.
 *   x: device double[n][3], m: device double[n], a: device double[n][3] out,
 *   phi: device double[n] out or NULL; eps >= 0; cuda_stream: cudaStream_t
 *   (NULL: the legacy default stream); the current device is used.
 * The i-particles keep the caller's order, so pair differences are formed
 * in double-float (FP32 offset plus its FP32 residual), accurate to FP32
 * relative to |d| however the particles are spread; eps = 0 gives a
 * coincident pair no contribution. If a device-side wait of the force
 * kernel gives up (bounded at two seconds), every output of the call is NaN.
 * Returns PG_EINVAL when n > PG_NOALLOC_MAX_N (or other bad arguments),
 * PG_ECUDA when a launch fails; asynchronous otherwise. The first call on a
 * device looks up the scratch array's device address: make it before any
 * stream capture. All calls share the one array, so calls that overlap on
 * the GPU race; order them on one stream. */
int pg_newton_allpairs_noalloc(const double *x, const double *m, long long n, double eps,
                               double *a, double *phi, void *cuda_stream);

/* Text of the last error of this context ("" if none); NULL ctx: last
 * error of pg_create. Valid until the next call on the context. */
const char *pg_last_error(pg_ctx *ctx);

/* Library version string. */
const char *pg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PG_H */
