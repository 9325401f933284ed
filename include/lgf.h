/*
 * lgf.h -- C ABI of a GB300 (sm_103a) library for the free-space 7-point Poisson solve and the
 * discrete heat-kernel (integrating-factor) apply on block-structured multi-level meshes, after
 * Yu, Dorschner & Colonius, "Multi-resolution lattice Green's function method for incompressible
 * flows" (J. Comput. Phys., 2020).
 *
 * Problem statement (Sec. 2.2, Eqs. (eq:discrete_laplace)-(eq:lgf_convolution)): on a lattice of
 * spacing h, L_h phi = f with phi -> 0 at infinity, L_h the 7-point Laplacian
 * h^-2 (sum_{+-e_i} phi(n +- e_i) - 6 phi(n)).  The unique decaying solution is the lattice
 * convolution phi = h^2 (G * f) with the lattice Green's function G (L_1 G = delta).  On a composite
 * mesh of levels k = 0..K-1 (h_k = h_0 / 2^k, level 0 coarsest, Sec. 3.1) the solve follows the
 * FLGF-AMR algorithm of Sec. 3.4 (Eqs. (eq:combine_S)-(eq:FLGF-AMR)); the heat apply follows
 * FIF-AMR, Sec. 3.5 (Eq. (eq:FIF-AMR)).
 *
 * Conventions shared by every call
 *  - Blocks are B^3 cells (B in {8, 16}).  Block (bx, by, bz) of level k holds the level-k cells
 *    B*(bx, by, bz) + [0, B)^3.  Field arrays are laid out [ncomp][sum_k nblocks_k][B][B][B]
 *    (blocks in mesh order, level 0 first; inside a block z slowest, x fastest).
 *  - Omega_k (the cells where level k holds the solution) is every cell of a level-k block that no
 *    level-(k+1) block covers; every level-(k+1) block must lie inside level-k blocks (nesting).
 *  - Pointers named *_dev are DEVICE pointers owned by the caller; pointers without the suffix are
 *    HOST pointers owned by the caller and only read during the call.
 *  - Every call is asynchronous on the given CUDA stream (NULL = the legacy default stream) unless
 *    documented otherwise; outputs are valid once the stream reaches the end of the call's work.
 *  - Status: 0 (LGF_OK) on success, a negative LGF_E_* otherwise.  Nothing is thrown across the ABI.
 *    lgf_last_error() returns a thread-local message for the last failing call of that thread.
 *    On error, output contents are unspecified.
 */
#ifndef LGF_H
#define LGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes */
#define LGF_OK 0
#define LGF_E_INVALID_ARG (-1)  /* null pointer, bad size, unsupported enum value */
#define LGF_E_MESH (-2)         /* mesh not nested, duplicate blocks, block size mismatch */
#define LGF_E_TABLE_RANGE (-3)  /* the table does not cover a block offset the mesh needs */
#define LGF_E_OOM (-4)          /* device allocation failed */
#define LGF_E_CUDA (-5)         /* a CUDA runtime call or kernel launch failed */
#define LGF_E_TIMEOUT (-6)      /* a bounded device-side wait gave up (batched scheduler) */
#define LGF_E_PRECISION (-7)    /* FP64 residual above opts->residual_tol */
#define LGF_E_UNSUPPORTED (-8)  /* valid request the library does not implement */

/* ---- storage types of caller fields */
#define LGF_F64 0
#define LGF_F32 1

/* ---- arithmetic of the convolution path
 *  FP64 : native double everywhere.
 *  FP32 : plain single precision (error ~1e-6 relative; reported, not a 1e-10 path).
 *  DF32 : "mixed": FP32 hardware, every value a pair of floats (hi + lo) with error-free products
 *         (fmaf) and sums, about 44 significant bits; the FP64 residual is the acceptance check. */
#define LGF_PREC_FP64 0
#define LGF_PREC_FP32 1
#define LGF_PREC_DF32 2

/* ---- how the per-frequency sum over block pairs is evaluated
 *  PAIR : direct sum over every (target, source) block pair with per-offset kernel spectra.
 *  BOX  : the same sum, diagonalised by a zero-padded FFT over each level's block grid.
 *  AUTO : the autotuner's choice from the pair count and grid fill. */
#define LGF_MAC_AUTO 0
#define LGF_MAC_PAIR 1
#define LGF_MAC_BOX 2

/* ---- table flags: which spectrum formats lgf_table_create keeps on the device */
#define LGF_TBL_FP64 1u
#define LGF_TBL_FP32 2u
#define LGF_TBL_DF32 4u
#define LGF_TBL_BOX_ONLY 8u  /* keep no per-offset spectra: only the block-index FFT mode is available
                                 (its spectra are built per box shape on first use) */

typedef struct lgf_table lgf_table; /* opaque: device LGF values + kernel spectra + workspaces */

typedef struct lgf_mesh {
  int32_t nlevels;            /* K >= 1 */
  int32_t block;              /* B, equal to the table's block size */
  double h0;                  /* level-0 spacing (> 0); h_k = h0 / 2^k */
  const int32_t *nblocks;     /* host [K]: blocks per level (>= 1 each) */
  const int32_t *block_ijk;   /* host [sum nblocks][3]: (bx, by, bz) per block, level by level */
  const uint8_t *block_role;  /* host [sum nblocks] or NULL (= all 3).  bit0: the block carries
                                 source values; bit1: the block receives output.  Honoured for
                                 K = 1; for K > 1 every block is both. */
  int32_t n_ext;              /* N_E >= 0: width in cells of the extended correction region
                                 Omega_k^E (Eq. (eq:extended_regions), max-norm, whole cells) */
} lgf_mesh;

typedef struct lgf_solve_opts {
  int32_t precision;     /* LGF_PREC_* */
  int32_t mac_mode;      /* LGF_MAC_* */
  int32_t residual;      /* 1: compute the FP64 residual into the report (synchronises) */
  int32_t timing;        /* 1: time the phases with CUDA events into the report (synchronises) */
  double residual_tol;   /* > 0 with residual = 1: LGF_E_PRECISION when residual_rel exceeds it */
  int32_t dft_slices;    /* 0: block-index DFT passes on the CUDA cores.  S > 0: those passes run as
                            tensor-core GEMMs (BF16 operands, FP32 accumulation) with S split-precision
                            digit slices per operand, exact per slice level and recombined in the
                            solve's arithmetic: FP32 takes S = 1..3 (1 = plain BF16), DF32 S = 4..6
                            (relative error of a pass about 2^-(7+8(S-1)) of each cell line's largest
                            value).  BOX mode only (AUTO picks BOX where the level allows it); FP64
                            rejects S > 0 with LGF_E_UNSUPPORTED. */
  int32_t flags;         /* OR of LGF_SOLVE_* (0 for the method as published) */
} lgf_solve_opts;

/* ---- lgf_solve_opts.flags
 *  NO_CORRECTION : multi-level solves without the source correction S psi_{k-1} of Eq. (eq:source_correct):
 *                  phi^k = P psi_{k-1} + L_k^{-1} sum_i P_{i->k} fhat_i (the uncorrected composite solve the
 *                  bump test of Sec. 3.4 compares against; single-level solves are unaffected). */
#define LGF_SOLVE_NO_CORRECTION 1

typedef struct lgf_report {
  double ms_total;        /* with timing = 1: wall time of the call's device work */
  double ms_phase[8];     /* restrict, correction, forward, mac, inverse, interp, residual, heat */
  double residual_rel;    /* max |L_k phi - source| / max |source| over interior output cells */
  int64_t target_cells;   /* cells written (sum over levels of |Omega_k| or target blocks) */
  int64_t source_blocks;  /* blocks forward-transformed, summed over levels and source sets */
  int64_t target_blocks;  /* blocks inverse-transformed */
  int64_t pairs;          /* block pairs summed by the PAIR mode (0 for BOX) */
  int64_t scratch_bytes;  /* device workspace held by the table for this stream */
  int64_t kernel_launches;/* kernels this call launched */
  int32_t mac_mode_used;  /* LGF_MAC_PAIR or LGF_MAC_BOX */
  int32_t reserved;
  /* method-minimum work of the call, independent of how the kernels realise it (Poisson solves):
   *   alg_bytes = sum over levels of ncomp (source cells + target cells) x (storage bytes of f, phi)
   *               + the unique kernel-spectrum values the level needs x (bytes of a real in the arithmetic)
   *               (block-index mode: the real spectrum of G is even in every axis, so (P_a B / 2 + 1) values
   *               per axis are unique; pair mode: (2B)^2 (B+1) complex values per block offset used);
   *   alg_flops = 5 M log2 M per complex FFT of M points (forward and inverse of every transformed field)
   *               plus 8 flops per complex multiply-add of the pair sums. */
  int64_t alg_bytes;
  double alg_flops;
} lgf_report;

/*
 * lgf_table_create -- tabulate the unit-lattice LGF and the kernel spectra (Sec. 5: the LGF is
 * evaluated once at start-up and stored).
 *   out              : receives the new table (caller destroys it with lgf_table_destroy).
 *   block            : B (8 or 16).
 *   max_block_offset : host [3]; spectra are kept for every block offset o with |o_a| <= this,
 *                      and G for every lattice offset up to B*(max+1) per axis.  A mesh level
 *                      whose block extent along axis a exceeds max_block_offset[a] + 1 (after
 *                      adding the blocks the solve needs around Omega_k^E) is rejected with
 *                      LGF_E_TABLE_RANGE.
 *   flags            : OR of LGF_TBL_*; the precisions a solve may use must be present.
 *   cuda_stream      : stream for the generation kernels; the call synchronises it before
 *                      returning, so the table is ready for use on any stream.
 * G(n) = -int_0^inf prod_i e^{-2t} I_{n_i}(2t) dt is computed in FP64 on the device (composite
 * Gauss-Legendre quadrature in ln t with the large-t Hankel tail).
 */
int lgf_table_create(lgf_table **out, int32_t block, const int32_t max_block_offset[3],
                     uint32_t flags, void *cuda_stream);

/*
 * lgf_table_prepare -- build everything a Poisson solve of mesh m on cuda_stream uses (the cached plan of
 * the mesh, the block-index FFT spectra of each level's box shape, the stream's workspace for ncomp
 * components of the given storage type and opts->precision / mac_mode) by one solve of a zero source into
 * trial fields it allocates and frees.  Afterwards solves of that mesh with those options on that stream
 * allocate nothing and only read the table (so solves on different streams, each prepared, may run
 * concurrently); without it the first solve does this work.  Synchronises cuda_stream.
 */
int lgf_table_prepare(lgf_table *t, const lgf_mesh *m, int32_t ncomp, int32_t dtype, const lgf_solve_opts *opts,
                      void *cuda_stream);

/* lgf_table_destroy -- release a table and every workspace it holds (synchronises the device). */
int lgf_table_destroy(lgf_table *t);

/*
 * lgf_table_lgf_values -- copy G on the lattice octant [0, n]^3 into host memory
 * (host_out[(c*(n+1) + b)*(n+1) + a] = G(a, b, c)); n must not exceed the table's lattice extent.
 * Synchronous.  For tests and diagnostics.
 */
int lgf_table_lgf_values(const lgf_table *t, int32_t n, double *host_out);

/*
 * lgf_poisson_solve -- free-space solve of L phi = f on the composite mesh (Sec. 3.4 FLGF-AMR:
 * cumulative coarsening of the sources, level-by-level convolution with the commutation source
 * correction S psi_{k-1} on Omega_k and Omega_k^E, interpolation of the coarser solution, and
 * restriction to Omega_k).
 *   ncomp   : number of independent scalar components (>= 1), e.g. 3 for a vector Poisson.
 *   f_dev   : device [ncomp][sum nblocks][B^3] source in `dtype`; values outside Omega_k (and of
 *             blocks without the source role) are ignored.
 *   phi_dev : device [ncomp][sum nblocks][B^3] output in `dtype`; written on Omega_k of blocks
 *             with the target role, left untouched elsewhere.  Must not alias f_dev.
 *   dtype   : LGF_F64 or LGF_F32 storage of f and phi (independent of opts->precision).
 *   opts    : may be NULL (FP64, AUTO, no residual, no timing).
 *   rep     : may be NULL.
 */
int lgf_poisson_solve(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev,
                      void *phi_dev, int32_t dtype, const lgf_solve_opts *opts, lgf_report *rep,
                      void *cuda_stream);

/*
 * lgf_heat_apply -- integrating-factor apply (Sec. 2.3 Eq. (eq:IF-single); Sec. 3.5 FIF-AMR):
 * g_k = Gamma_k [ E_{alpha_k} * (P_k fhat) ] with E_alpha(n) = prod_i e^{-2 alpha} I_{|n_i|}(2 alpha),
 * alpha_k = alpha_finest * 4^{-(K-1-k)} (Eq. (eq:composite-LGF-IF)), P_k fhat the reconstruction of
 * the AMR data on level k (own values, interpolation from coarser, coarsening from finer levels).
 *   t            : may be NULL (the heat kernel needs no LGF table); when non-NULL its workspace
 *                  pool is used.
 *   alpha_finest : kappa*dt/h_finest^2 >= 0.
 *   f_dev, g_dev : as for lgf_poisson_solve; g written on Omega_k.
 * Only opts->precision (FP64, FP32 or DF32: the arithmetic of the convolution sums) and opts->timing
 * are read.
 */
int lgf_heat_apply(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev,
                   void *g_dev, int32_t dtype, double alpha_finest, const lgf_solve_opts *opts,
                   lgf_report *rep, void *cuda_stream);

/*
 * lgf_velocity_refresh -- velocity from vorticity on one level (Sec. 4.1, Eq. (eq:vel_update)):
 * u = -C^T L_E^{-1} omega.  Staggered lattice (Sec. 2.1): component a of cell n is stored at index n,
 * the velocity at the face centre n + (1,1,1)/2 + e_a/2, the vorticity (and the streamfunction) at the
 * edge centre n + (1,1,1) - e_a/2 (in cells).  L_E^{-1} is the free-space LGF solve of each edge
 * component; C^T (= the edge-to-face curl, the transpose of the face-to-edge curl C, Eq. (eq:mimetic)) is
 *   (C^T psi)_x[n] = (psi_z[n] - psi_z[n - e_y] - psi_y[n] + psi_y[n - e_z]) / h, and cyclically.
 *   m            : one level (nlevels = 1); block_role is ignored: every block is a source and receives
 *                  u.  The streamfunction is solved on the blocks and on their -x, -y, -z
 *                  neighbour blocks, so the table's max_block_offset must cover the box extended by one
 *                  block toward -x, -y and -z.
 *   omega_dev    : device [3][nblocks][B^3] (x fastest) in dtype; read only.
 *   u_dev        : device [3][nblocks][B^3] in dtype; every cell written.
 *   opts, rep    : as for lgf_poisson_solve (the report is the streamfunction solve's, with the curl
 *                  kernel added to kernel_launches).
 * Scratch: the vorticity and the streamfunction on the extended block set, allocated and freed in
 * stream order.  Errors: as lgf_poisson_solve; LGF_E_MESH for nlevels != 1; LGF_E_OOM for the scratch.
 */
int lgf_velocity_refresh(lgf_table *t, const lgf_mesh *m, const void *omega_dev, void *u_dev, int32_t dtype,
                         const lgf_solve_opts *opts, lgf_report *rep, void *cuda_stream);

/*
 * lgf_stage_projection -- the pressure projection of one half-explicit Runge-Kutta stage on the AMR grid
 * (Sec. 2.4, Eqs. (eq:projection-1), (eq:projection-2); Sec. 3.6, Eqs. (eq:approx0)-(eq:approx4)):
 *     L_C p = D r,    u = H (r - G p),     H = the integrating factor E_alpha of lgf_heat_apply.
 * Staggered lattice (Sec. 2.1): component a of a face field (r, u) at cell n is stored at index n and sits on
 * the face n + (1/2, 1/2, 1/2) + e_a / 2; p sits at the cell centre.  D r(n) = sum_a (r_a[n] - r_a[n - e_a]) / h,
 * (G p)_a[n] = (p[n + e_a] - p[n]) / h, so D G = L_C (Eq. (eq:mimetic)).  On the AMR grid:
 *     D^r   = D (P_k r^) on Omega_k, P_k r^ the level-k reconstruction (own values on Omega_k, interpolation
 *             of coarser and 8-child means of finer levels, each component as a cell-centred scalar), which
 *             supplies the faces across the Omega_k boundary (the one-cell-larger restriction of Sec. 3.6);
 *     p^    = FLGF-AMR(D^r) on Omega_k (lgf_poisson_solve);
 *     w^    = r^ - G (P_k p^) on Omega_k;
 *     u^    = FIF-AMR(w^) (lgf_heat_apply with alpha_finest).
 * Fields outside the AMR grid are zero (the computational domain's truncation, Sec. 4.1).
 *   r_dev        : device [3][sum nblocks][B^3] in dtype, read on Omega_k.
 *   u_dev        : device [3][sum nblocks][B^3] in dtype, written on Omega_k.
 *   p_dev        : device [1][sum nblocks][B^3] in dtype or NULL; receives p^ on Omega_k when given.
 *   alpha_finest : kappa (c~_i - c~_{i-1}) dt / dx_finest^2 of the stage (Eq. (eq:composite-LGF-IF)).
 *   opts         : precision / mac_mode / flags of the Poisson solve and the arithmetic of the IF; may be NULL.
 * block_role is ignored (every block carries r and receives u).  Scratch (D^r, p^, w^) is held by the table
 * per stream.  Errors: as lgf_poisson_solve and lgf_heat_apply.
 */
int lgf_stage_projection(lgf_table *t, const lgf_mesh *m, const void *r_dev, void *u_dev, void *p_dev, int32_t dtype,
                         double alpha_finest, const lgf_solve_opts *opts, lgf_report *rep, void *cuda_stream);

/*
 * lgf_refinement_indicator -- the Poisson solve of lgf_poisson_solve together with the refinement
 * indicator of the adaptive mesh (Sec. 4.2, Eqs. (eq:refine1), (eq:maximumS), (eq:refine2)), reduced on
 * the device from the combined source the solve builds anyway (Eq. (eq:combined_source)):
 *   S_k = S psi_{k-1} + sum_{i >= k} P_{i->k} fhat_i   (the correction source on Omega_k and Omega_k^E plus
 *         the level's own and the coarsened finer sources; S_0 = the cumulative source F_0),
 *   |S_k| = Euclidean norm over the ncomp components,
 *   rms   = sqrt(mean over the B^3 cells of a caller block of |S_k|^2),
 *   S_max = max(previous S_max, largest block rms over all levels)               (Eq. (eq:maximumS)),
 *   refine (bit 0)  : |S_k| > alpha^(N_l - k) S_max at a cell of the block        (Eq. (eq:refine1)), or at an
 *                     Omega_{k+1}^E cell outside the level-(k+1) blocks that lies in this block,
 *   coarsen (bit 1) : |S_k| < beta alpha^(N_l - k) S_max at every cell of the block (Eq. (eq:refine2)).
 *   t, m, ncomp, f_dev, phi_dev, dtype, opts, rep : as for lgf_poisson_solve; every level (also a single
 *                  one) runs the composite-mesh driver, so block_role is ignored.
 *   ind          : host struct, read during the call; its three device pointers are written in stream
 *                  order (s_max_dev is read first: pass 0 at the first step, then keep the value).
 * Errors: as lgf_poisson_solve; LGF_E_INVALID_ARG for a NULL or out-of-range indicator field,
 * LGF_E_UNSUPPORTED above 16 levels.
 */
typedef struct lgf_indicator {
  double alpha;          /* 0 < alpha < 1 */
  double beta;           /* 0 < beta < 1 */
  int32_t n_levels_max;  /* N_l, the prescribed maximum level index (>= nlevels - 1) */
  int32_t reserved;      /* 0 */
  double *rms_dev;       /* device [sum nblocks]: block RMS of |S_k|, caller block order */
  uint8_t *flags_dev;    /* device [sum nblocks]: bit 0 refine, bit 1 coarsen */
  double *s_max_dev;     /* device [1], in/out: S_max carried over time */
} lgf_indicator;
int lgf_refinement_indicator(lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev, void *phi_dev,
                             int32_t dtype, const lgf_solve_opts *opts, const lgf_indicator *ind, lgf_report *rep,
                             void *cuda_stream);

/*
 * lgf_device_status -- synchronise the device and read the table's device status word: LGF_E_TIMEOUT
 * (and the word cleared) when a bounded device-side wait of a kernel that used this table gave up since
 * the last read, else LGF_OK.  Solves with opts->timing or opts->residual set read it themselves.
 */
int lgf_device_status(lgf_table *t);

/*
 * lgf_selftest_wait_timeout -- launch one CTA that waits on an mbarrier no thread ever arrives at, with
 * the bounded wait of the tensor-core kernels limited to 2^log2_cycles SM cycles (10..31).  The wait
 * gives up, the kernel sets the table's status word and returns; a following lgf_device_status reports
 * LGF_E_TIMEOUT and clears it.  Checks the timeout path without faulting or hanging the GPU.
 */
int lgf_selftest_wait_timeout(lgf_table *t, int32_t log2_cycles, void *cuda_stream);

/* ---- batches: many independent instances solved as one unit, capturable into a CUDA graph */
typedef struct lgf_batch lgf_batch; /* opaque */

/*
 * lgf_batch_create -- plan a batch of `ninst` independent composite-mesh problems sharing table `t`
 * (the right-hand sides of the stages of a half-explicit Runge-Kutta step, Sec. 2.4: one Poisson
 * solve, Eq. (eq:projection-1), and one integrating-factor apply, Eq. (eq:projection-2), per instance).
 *   meshes   : host [ninst]; copied (the caller's arrays may be released after the call).  block_role
 *              is ignored; every mesh's block size must equal the table's.
 *   ncomp    : components per instance; dtype: LGF_F64 / LGF_F32 storage of every field.
 *   alpha    : host [ninst] integrating-factor argument kappa*dt/h_finest^2 per instance, or NULL (0).
 *   opts     : precision / mac_mode for every solve (residual and timing are forced off); may be NULL.
 *   nstreams : 1..64 internal streams; instances are dealt longest-first to the least-loaded stream.
 */
int lgf_batch_create(lgf_batch **out, lgf_table *t, int32_t ninst, const lgf_mesh *meshes, int32_t ncomp,
                     int32_t dtype, const double *alpha, const lgf_solve_opts *opts, int32_t nstreams);
int lgf_batch_destroy(lgf_batch *b);

/*
 * lgf_batch_stage -- for every instance i: phi_dev[i] = L^{-1} f_dev[i] and, when g_dev is non-NULL,
 * g_dev[i] = FIF-AMR heat apply of f_dev[i].  Device arrays laid out as for lgf_poisson_solve.
 *   alpha : host [ninst] integrating-factor argument of this stage per instance, or NULL for the
 *           values given at create time.  A HERK stage i uses (c~_i - c~_{i-1}) dt kappa / dx_finest^2
 *           (Eq. (eq:composite-LGF-IF) with the tableau of Table tab:HREK), so it changes from stage to stage.
 * Work runs on the batch's streams, forked from and joined back into cuda_stream (asynchronous).
 */
int lgf_batch_stage(lgf_batch *b, const void *const *f_dev, void *const *phi_dev, void *const *g_dev,
                    const double *alpha, void *cuda_stream);

/*
 * lgf_batch_graph_create -- run the stages once eagerly (building every plan, spectrum and workspace),
 * then capture `nstages` chained stages into a CUDA graph.  With g_dev non-NULL: stage 0 reads f and
 * writes g, stage s >= 1 reads the previous stage's heat output (g or tmp, alternating) and writes the
 * other; every stage writes phi.  With g_dev NULL every stage is the Poisson solve phi = L^{-1} f alone
 * (tmp_dev unused).  alpha_stages: host [nstages][ninst] per-stage integrating-factor arguments, or NULL
 * for the create-time values.  cuda_stream must be a non-default stream.  Synchronises.
 * lgf_batch_graph_launch replays it with one cudaGraphLaunch; lgf_batch_graph_nodes returns its node count.
 */
int lgf_batch_graph_create(lgf_batch *b, int32_t nstages, const void *const *f_dev, void *const *phi_dev,
                           void *const *g_dev, void *const *tmp_dev, const double *alpha_stages,
                           void *cuda_stream);
int lgf_batch_graph_launch(lgf_batch *b, void *cuda_stream);

/*
 * lgf_batch_graph_create_io -- capture one Poisson stage (phi = L^{-1} f per instance, Sec. 3.4) with its
 * host transfers inside the graph: f_host[i] -> f_dev[i] on a copy-in stream in the order the solves start,
 * each solve waiting for its own source only, and phi_dev[i] -> phi_host[i] on a copy-out stream after the
 * solve, in the order the solves are expected to end, so the copies overlap the other instances' solves.
 *   f_host, phi_host : host [ninst] pointers to PINNED host buffers (cudaHostAlloc or cudaHostRegister),
 *                      each the instance's field bytes (ncomp x its blocks x B^3 x 8 or 4 for the dtype);
 *                      pageable memory is rejected with LGF_E_INVALID_ARG.  Owned by the caller.
 *   f_dev, phi_dev   : host [ninst] device buffers of the same sizes (the staging copies).
 * Runs the stage once eagerly (copies included), then captures; synchronises.  lgf_batch_graph_launch
 * replays it; phi_host holds the results once cuda_stream reaches the end of the replay.
 */
int lgf_batch_graph_create_io(lgf_batch *b, const void *const *f_host, void *const *phi_host,
                              const void *const *f_dev, void *const *phi_dev, void *cuda_stream);

/*
 * lgf_batch_autotune -- measure and choose how the batch runs (the batched solver's autotuner):
 *   (i)  per instance, the evaluation of its block-index DFT passes: the CUDA-core conjugate-pair passes or,
 *        for DF32 / FP32 solves, the tensor-core DFT-GEMM with 5 / 3 digit slices (the fewest that keep the
 *        arithmetic's accuracy), whichever solves the instance faster (three timed solves each);
 *   (ii) the instance order, longest measured solve first, dealt to the least-loaded stream;
 *   (iii) the stream count from {1, 2, 4, 8, 16, 32} (at most ninst), by timing a Poisson stage captured
 *        into a graph and replayed (the fastest of five replays; eager stages when cuda_stream cannot
 *        capture, e.g. the legacy default stream); a larger count is taken only when it is at least 1 %
 *        faster.
 * f_dev / phi_dev: the instances' fields (phi is overwritten).  Synchronises cuda_stream.  A graph captured
 * before the call keeps the old choices; capture after it.
 */
int lgf_batch_autotune(lgf_batch *b, const void *const *f_dev, void *const *phi_dev, void *cuda_stream);

/* lgf_batch_tuning -- the choices: stream count, per-instance digit slices (0 = CUDA-core passes) and measured
 * solve time in ms (0 before lgf_batch_autotune).  Each output pointer may be NULL; slices and ms hold ninst. */
int lgf_batch_tuning(const lgf_batch *b, int32_t *nstreams, int32_t *slices, double *ms);
int lgf_batch_graph_nodes(const lgf_batch *b, int64_t *nodes);

/*
 * lgf_poisson_solve_static -- single-level solve (pair mode) that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that must not allocate during a
 * solve (a device-memory budget fixed at start-up, or a thread that must not block on the
 * allocator, which may synchronise the device).  Its scratch is a file-scope device array of
 * LGF_STATIC_SCRATCH_BYTES = 32 MiB that every GPU loading the library reserves until exit.
 *   t, m, ncomp, f_dev, phi_dev, dtype : as for lgf_poisson_solve (m->nlevels must be 1).
 *   precision   : LGF_PREC_FP64, LGF_PREC_FP32 or LGF_PREC_DF32 (the table must hold its spectra).
 *   cuda_stream : stream of the work.
 * Requests whose scratch (source and target spectra: ncomp x blocks x (2B)^2 (B+1) complex values,
 * plus index lists) exceeds 32 MiB fail with LGF_E_INVALID_ARG and a message giving the size.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Every call copies its block index lists from pageable host
 * memory into the array; on a stream that is capturing, the call returns LGF_E_UNSUPPORTED before
 * enqueueing anything, and a failed copy returns LGF_E_CUDA.  All calls share the array: calls whose
 * GPU work may overlap race on it and must be ordered by the caller.  It calls no cudaMalloc/cudaFree.
 */
int lgf_poisson_solve_static(const lgf_table *t, const lgf_mesh *m, int32_t ncomp, const void *f_dev,
                             void *phi_dev, int32_t dtype, int32_t precision, void *cuda_stream);

/* lgf_last_error -- message for the last non-zero status returned on the calling thread. */
const char *lgf_last_error(void);

/* lgf_version -- library version string. */
const char *lgf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LGF_H */
