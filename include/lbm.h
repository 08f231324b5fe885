/*
 * lbm.h - C ABI of the GB300 elastic-wall D3Q19 lattice Boltzmann library.
 *
 * One call advances a compacted sparse vascular lattice by LBGK timesteps
 * (Sec. 2.1, Eq. LBE_SRT) with the paper's localised elastic wall (Sec. 2.3:
 * Guo-Zheng-Shi wall with Delta = 1 and wall velocity
 * U_w = (F + dr - dx)/dr U_f; Sec. 2.4: tube law dE = (1 - sigma^2) R^2/(Y h)
 * (p - P0)), the rigid bounce-back wall it is compared with (Sec. 2.4), a
 * velocity-profile inlet and fixed-density outlets (Sec. 3).
 *
 * Conventions shared by every entry point:
 *   - Return value: LBM_OK (0) or a negative LBM_E* status.  No call aborts
 *     the process; lbm_last_error(ctx) gives a one-line message.
 *   - Host arrays passed in are copied before the call returns; the caller
 *     keeps ownership.  Output arrays are written, never retained.
 *   - Sites are numbered in canonical order: ascending (x*ny + y)*nz + z over
 *     the fluid voxels (z fastest).  Directions follow the canonical D3Q19
 *     order: 0 rest; 1/2 +-x; 3/4 +-y; 5/6 +-z; 7/8 (+1,+1,0)/(-1,-1,0);
 *     9/10 (+1,-1,0)/(-1,+1,0); 11/12 (+1,0,+1)/(-1,0,-1);
 *     13/14 (+1,0,-1)/(-1,0,+1); 15/16 (0,+1,+1)/(0,-1,-1);
 *     17/18 (0,+1,-1)/(0,-1,+1).
 *   - Device memory comes from the caller's allocator (or cudaMalloc when it
 *     is NULL) and is released by lbm_destroy.  All work is ordered on the
 *     CUDA stream given at build time (lbm_set_stream changes it); inside a
 *     step the boundary kernel runs on a private stream forked from and
 *     joined back into that stream.
 *   - One context per host thread; contexts share no state.
 *   - Device-side faults of the method (non-finite or non-positive density)
 *     are sticky flags reported by lbm_sync as LBM_EUNSTABLE.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Device allocator hook: alloc returns device memory of at least `bytes`
 * bytes (256-byte aligned) or NULL; free releases it.  `user` is passed back. */
typedef struct lbm_allocator {
  void *(*alloc)(size_t bytes, void *user);
  void (*free)(void *ptr, void *user);
  void *user;
} lbm_allocator;

/* An inlet or outlet (Sec. 3).  Ghost voxels labelled 2+k belong to iolet k.
 *   kind     LBM_IOLET_VELOCITY: the boundary population is rebuilt by the
 *            GZS rule from (rho_f, u_in(x, n)); LBM_IOLET_DENSITY: from
 *            (rho, u_f) (fixed-pressure outlet, p = c_s^2 rho, Eq. Pressure).
 *   u_in(x, n) = axis * (u_mean p0(r) + u_amp (ps(r) sin(th) + pc(r) cos(th))),
 *            th = 2 pi n / period + phase (period <= 0: steady, u_amp unused),
 *            r = distance of the fluid site x from the line (centre, axis).
 *   profile  LBM_PROFILE_PARABOLIC: p0 = ps = 2 (1 - r^2/radius^2)+, pc = 0;
 *            LBM_PROFILE_WOMERSLEY: p0 parabolic, ps + i pc = the rigid-tube
 *            Womersley shape (Sec. 2.2 with M = 1) at alpha = radius
 *            sqrt(2 pi / period / nu), nu = (tau - 1/2)/3, unit mean over the
 *            disc, zero outside it; LBM_PROFILE_PLUG: p0 = ps = 1, pc = 0.
 *   axis     flow direction (normalised by the library); for a density iolet
 *            it only orients the reported flux. */
typedef struct lbm_iolet {
  int32_t kind;
  int32_t profile;
  double rho;
  double u_mean, u_amp, period, phase;
  double centre[3], axis[3], radius;
} lbm_iolet;

enum {
  LBM_OK = 0,
  LBM_EINVAL = -1,    /* invalid argument or inconsistent input */
  LBM_ENOMEM = -2,    /* the allocator (or host malloc) failed */
  LBM_ECUDA = -3,     /* a CUDA runtime call failed; see lbm_last_error */
  LBM_EUNSTABLE = -4, /* a kernel saw a non-finite or non-positive density */
  LBM_ETIMEOUT = -5,  /* a bounded device wait gave up */
  LBM_ESTATE = -6,    /* call not valid in the context's current state */
  LBM_ECHECK = -7     /* checked builds only (-DLBM_CHECKED): a neighbour or slot index out of
                         range, or a population slot not written exactly once in a step */
};

/* Population storage.  Every variant stores f_i - w_i (the deviation from the
 * rest equilibrium), so that the stored value keeps its significant bits
 * (essential for the 16-bit *S variants, a free accuracy gain for the others). */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 };
enum { LBM_WALL_BOUNCEBACK = 0, LBM_WALL_ELASTIC_GZS = 1 };
enum { LBM_IOLET_VELOCITY = 0, LBM_IOLET_DENSITY = 1 };
enum { LBM_PROFILE_PARABOLIC = 0, LBM_PROFILE_WOMERSLEY = 1, LBM_PROFILE_PLUG = 2 };

/* lbm_build_lattice - compact the fluid voxels and build the link tables
 * (the sparse lattice of Sec. 1; D3Q19 links of Sec. 2.1).
 *   labels     host uint8 [nx*ny*nz], index (x*ny + y)*nz + z: 0 solid,
 *              1 fluid, 2+k ghost of iolet k (k < n_iolets).  A link to a
 *              solid voxel or out of the box is a wall link; a link to a
 *              ghost of iolet k is an iolet link.
 *   iolets     host [n_iolets] (copied).
 *   storage    LBM_F64 / LBM_F32 / LBM_F16S / LBM_BF16S.  Collision runs in
 *              FP64 for LBM_F64 and in FP32 otherwise; the wall's tube-law
 *              update always runs in FP64.
 *   tau        relaxation time, > 1/2 (Eq. LBE_SRT).
 *   alloc      device allocator, or NULL for cudaMalloc/cudaFree.
 *   cuda_stream  cudaStream_t for every kernel and copy (NULL = legacy stream).
 *   out        receives the context.  Populations start at rest (rho = 1,
 *              u = 0), wall model bounce-back, step counter 0.
 * Errors: LBM_EINVAL for bad sizes, tau <= 1/2, a label >= 2 + n_iolets, a
 * bad iolet (kind/profile out of range, zero axis, radius <= 0 for a profiled
 * inlet) or a fluid site touching two different velocity inlets; LBM_ENOMEM;
 * LBM_ECUDA. */
int lbm_build_lattice(const uint8_t *labels, int32_t nx, int32_t ny, int32_t nz,
                      const lbm_iolet *iolets, int32_t n_iolets, int32_t storage, double tau,
                      const lbm_allocator *alloc, void *cuda_stream, lbm_ctx **out);

/* lbm_set_wall_params - choose the wall rule and its per-wall-site parameters.
 *   wall_model  LBM_WALL_BOUNCEBACK (Sec. 2.4, half-way bounce-back) or
 *               LBM_WALL_ELASTIC_GZS (Sec. 2.3-2.4).
 *   rho0        reference density: p - P0 = c_s^2 (rho_f - rho0).
 *   F, kappa    host [n] in wall-site order (the sites with at least one wall
 *               link, ascending), or n == 1 to broadcast one value.  F is the
 *               velocity ratio U_R/U_f; kappa is the tube-law coefficient
 *               (1 - sigma^2) r0^2/(E h) in lattice units, so that at each
 *               step dE = kappa max(0, p - P0), dr = 1 + dE and
 *               U_w = (F + dr - 1)/dr u_f.  NULL means 0.
 * Errors: LBM_EINVAL for an unknown model, n not in {1, n_wall_sites}, or a
 * negative / non-finite F or kappa. */
int lbm_set_wall_params(lbm_ctx *ctx, int32_t wall_model, double rho0, const double *F,
                        const double *kappa, int64_t n);

/* lbm_init_fields - set f = f^eq(rho, u) (Eq. feq) at every site and reset the
 * step counter to 0.  rho host [n_sites] or NULL (1); u host [n_sites][3] or
 * NULL (0). */
int lbm_init_fields(lbm_ctx *ctx, const double *rho, const double *u);

/* lbm_step - enqueue n_steps >= 0 timesteps on the context's stream and
 * return without waiting.  Step n evaluates the inlet time factor at n. */
int lbm_step(lbm_ctx *ctx, int64_t n_steps);

/* lbm_step_diag - lbm_step of n_steps >= 1 timesteps whose last step also
 * reduces the diagnostics of the state it reads (the state after n_steps - 1
 * steps), as lbm_reduce defines them: out[0] total mass sum_x rho_x,
 * out[1 + k] the flux of rho u along iolet k's axis over the sites with a
 * link into it.  The step kernels add each tile's rho - 1 in FP32 (one value
 * per 32 sites) and write the momenta of the iolet sites; one more kernel adds
 * those in FP64 in a fixed order, so no extra pass over the populations is
 * made (Sec. 2.1 moments; the mass and flux sums of the benchmark contract).
 * out is a host array [1 + n_iolets].  The final sums and the copy into out
 * run on a stream of the library's own, ordered after this step and beside
 * the steps queued after it (two buffer sets used in turn); they are
 * complete after the next call that waits (lbm_sync, lbm_reduce,
 * lbm_moments to host memory, ...); page-locked memory keeps the copy
 * asynchronous.  The first call
 * allocates the device tables (a double per tile, three doubles per lane
 * of the tiles with iolet sites).  Errors: LBM_EINVAL (n_steps < 1, NULL
 * arguments), LBM_ENOMEM, LBM_ECUDA. */
int lbm_step_diag(lbm_ctx *ctx, int64_t n_steps, double *out);

/* lbm_moments - rho [n_sites] and u [n_sites][3] (FP64, canonical order) of
 * the current pre-collision state (Eqs. Density, Momentum).  Either pointer may
 * be NULL.  dst_is_device != 0: device pointers, written asynchronously on the
 * context's stream; 0: host pointers, the call waits for the copy. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, int32_t dst_is_device);

/* lbm_sync - wait for the context's stream; return LBM_EUNSTABLE if any kernel
 * since the last lbm_sync saw a non-finite or non-positive density (the flag
 * is then cleared), LBM_ECUDA on a CUDA error, else LBM_OK. */
int lbm_sync(lbm_ctx *ctx);

/* lbm_plan_lattice - the host half of lbm_build_lattice alone: the same
 * validation and compaction on the host, no GPU and no context, returning the
 * sizes the build would produce in out[8] (host): n_sites, n_wall_sites,
 * n_wall_links, n_tiles, bulk tiles, coherent boundary tiles, irregular
 * tiles, sites in bulk tiles (as lbm_info).  Errors as lbm_build_lattice,
 * message via lbm_last_error(NULL). */
int lbm_plan_lattice(const uint8_t *labels, int32_t nx, int32_t ny, int32_t nz,
                     const lbm_iolet *iolets, int32_t n_iolets, double tau, int64_t out[8]);

/* lbm_info - sizes of the context:
 *   out[0] n_sites, [1] n_wall_sites, [2] n_wall_links, [3] n_tiles (32 sites),
 *   [4] bulk tiles, [5] uniform boundary tiles, [6] irregular tiles,
 *   [7] step counter, [8] storage, [9] n_iolets, [10] device bytes held,
 *   [11] sites in bulk tiles. */
int lbm_info(const lbm_ctx *ctx, int64_t out[12]);

/* lbm_profile - when enable != 0, lbm_step records CUDA events on the
 * context's stream around each step: before the boundary kernel is forked to
 * the library's side stream, after the bulk kernel, and after the join.
 * lbm_profile_read waits, returns the summed device time of the steps
 * (ms[0], both kernels) and of the bulk kernel (ms[1]) and the launch counts
 * of the bulk (launches[0]) and boundary (launches[1]) kernels, then clears
 * the record.  Measurement only: no work is skipped. */
int lbm_profile(lbm_ctx *ctx, int32_t enable);
int lbm_profile_read(lbm_ctx *ctx, double ms[2], int64_t launches[2]);

/* lbm_export_lattice - the integer lattice (host arrays, any may be NULL):
 *   coords [n_sites][3] int32 voxel coordinates;
 *   nbr [n_sites][18] int32 neighbour along directions 1..18: site id >= 0,
 *     -1 wall, -2-k iolet k;
 *   wall_sites [n_wall_sites] int64 ascending;
 *   wall_links [n_wall_links][2] int64 (site, direction) sorted. */
int lbm_export_lattice(const lbm_ctx *ctx, int32_t *coords, int32_t *nbr, int64_t *wall_sites,
                       int64_t *wall_links);

/* lbm_wall_state - per wall site (wall-site order) the expansion dE and the
 * wall velocity U_w [n][3] computed by the most recent step (host arrays, any
 * may be NULL; zeros before the first step or under bounce-back).  Waits for
 * the stream. */
int lbm_wall_state(lbm_ctx *ctx, double *dE, double *Uw);

/* lbm_reduce - FP64 diagnostics of the current state, deterministic order:
 *   out[0] total mass sum_x rho_x;
 *   out[1 + k] sum over the sites with a link into iolet k of (rho u).axis_k.
 * out is a host array [1 + n_iolets]; the call waits for the stream. */
int lbm_reduce(lbm_ctx *ctx, double *out);

/* lbm_reduce_noalloc - the same diagnostics as lbm_reduce, for callers that
 * must not allocate device memory during the call (for example a monitoring
 * hook that runs while another component's memory pool owns the whole device,
 * where cudaMalloc can fail or force the pool to shrink, or a latency-bound
 * loop that cannot take the synchronisation cudaMalloc/cudaFree may cause).
 * The paper has no counterpart: this is a property of the library, not of the
 * method.  Scratch (1024 partial sums and up to 256 outputs, 10 KiB) lives in
 * a fixed device array that every GPU loading the library holds until the
 * process exits; the call itself allocates nothing.
 *   out            [1 + n_iolets] doubles, laid out as for lbm_reduce;
 *   out_is_device  != 0: out is device memory, written asynchronously on the
 *                  context's stream; 0: out is host memory, the call waits.
 * The first call on a device looks up the array's device address (with the
 * context's device current) and caches it for that CUDA context (a device
 * reset or a new primary context makes the next call look it up again); make
 * that first call before any stream capture.  All calls share the array, so
 * calls that overlap on the GPU race; serialise them (one stream, or wait
 * between calls).
 * Errors: LBM_EINVAL for NULL arguments or more than 255 iolets (beyond the
 * array); LBM_ECUDA. */
int lbm_reduce_noalloc(lbm_ctx *ctx, double *out, int32_t out_is_device);

/* lbm_get_populations / lbm_set_populations - the pre-collision populations
 * f[n_sites][19] (FP64, canonical site order, canonical directions),
 * converting to or from the in-place storage layout.  set also sets the step
 * counter.  *_is_device selects device (asynchronous) or host (waits)
 * pointers. */
int lbm_get_populations(lbm_ctx *ctx, double *f, int32_t dst_is_device);
int lbm_set_populations(lbm_ctx *ctx, const double *f, int64_t step, int32_t src_is_device);

/* Checkpoint of the exact device state (raw storage plus step counter), so a
 * resumed run is bit-identical to an uninterrupted one. */
size_t lbm_checkpoint_bytes(const lbm_ctx *ctx);
int lbm_checkpoint_save(lbm_ctx *ctx, void *host_buf, size_t bytes);
int lbm_checkpoint_load(lbm_ctx *ctx, const void *host_buf, size_t bytes);

/* lbm_wss - wall shear stress at m sites (a metric; the paper's WSS fields
 * are not defined there): sigma = -(1 - 1/(2 tau)) sum_i f_i^neq c_i c_i,
 * t = sigma n, WSS = |t - (t.n) n| for the given unit normals.
 *   sites host int64 [m] canonical ids; normals host [m][3]; out host [m]. */
int lbm_wss(lbm_ctx *ctx, const int64_t *sites, const double *normals, int64_t m, double *out);

/* ---------------------------------------------------------------- ensembles
 * An ensemble advances many independent lattices (members) together: each
 * timestep is one launch of the bulk kernel and one of the boundary kernel
 * covering the tiles of every member, so that many small vessels with their
 * own tau, F, kappa, inlet and outlet fill the GPU together.  The paper runs
 * one geometry at a time; this batching has no counterpart there.
 *
 * lbm_ensemble_create - members: [n] contexts built by lbm_build_lattice, all
 *   with the same storage, on the same device, at the same step; they stay
 *   owned by the caller and must outlive the ensemble.  The ensemble runs on
 *   private streams, ordered after the work already queued on the members'
 *   streams and before their later work.  Wall parameters set on a member with
 *   lbm_set_wall_params are picked up by the next lbm_ensemble_step.
 * lbm_ensemble_step - enqueue n_steps timesteps of every member and advance
 *   their step counters.  With LBM_TUNE_GRAPH_STEPS = G > 0 (even), whole
 *   blocks of G steps replay a CUDA graph captured on first use (the inlet
 *   time reads a device step counter, so replays stay exact).
 * lbm_ensemble_sync - wait, then lbm_sync every member (first error wins).
 * lbm_ensemble_tune - schedule knobs (chosen by an autotuner in the binding):
 *   LBM_TUNE_PREFETCH    L2 prefetch distance in tiles (>= 0);
 *   LBM_TUNE_SCHEDULE    0: members in the given order, 1: largest first;
 *   LBM_TUNE_GRAPH_STEPS steps per captured graph (even, 0 = direct launches);
 *   LBM_TUNE_PERSISTENT  1: each lbm_ensemble_step is one cooperative launch of a
 *                        persistent kernel whose CTAs take chunks of tiles from a
 *                        device counter and meet at a grid barrier after every
 *                        step (graphs are not used then); a barrier that does not
 *                        complete within ~1 s makes every CTA return and
 *                        lbm_ensemble_sync report LBM_ETIMEOUT;
 *   LBM_TUNE_BARRIER_EXTRA fault injection for tests: the grid barrier waits for
 *                        this many arrivals that never come (default 0), so a
 *                        persistent step times out instead of completing;
 *   LBM_TUNE_BULK_SITES  sites per lane of the bulk kernel: 1 (a 32-site tile per
 *                        warp), or two tiles per warp with two sites per lane and
 *                        FP32 pair arithmetic (FP32 and 16-bit storage; FP64
 *                        ignores it), the pairs being either two z-adjacent sites
 *                        of one tile (one packed load or store per direction
 *                        where the offset is even) or the same lane of both
 *                        tiles (scalar, aligned accesses; one address when the
 *                        second tile follows the first with the same offsets):
 *                        2 = adjacent sites on even steps, two tiles on odd
 *                        steps; 3 = adjacent sites on both; 4 = two tiles on
 *                        both.  Default: 2 for 16-bit storage, 1 otherwise;
 *   LBM_TUNE_BULK_WARPS  warps (tiles, or tile pairs) per CTA of the bulk
 *                        kernel: 4 (default) or 8, the same warps per SM.
 * Before using a member's own calls (moments, wall state, ...) call
 * lbm_ensemble_sync.  Errors: LBM_EINVAL (bad arguments, mixed storage or
 * steps), LBM_ESTATE (members drifted apart), LBM_ENOMEM, LBM_ECUDA; the
 * message is lbm_ensemble_last_error. */
typedef struct lbm_ensemble lbm_ensemble;
enum {
  LBM_TUNE_PREFETCH = 0,
  LBM_TUNE_SCHEDULE = 1,
  LBM_TUNE_GRAPH_STEPS = 2,
  LBM_TUNE_PERSISTENT = 3,
  LBM_TUNE_BARRIER_EXTRA = 4,
  LBM_TUNE_BULK_SITES = 5,
  LBM_TUNE_BULK_WARPS = 6
};
int lbm_ensemble_create(lbm_ctx *const *members, int32_t n, lbm_ensemble **out);
int lbm_ensemble_step(lbm_ensemble *ens, int64_t n_steps);
int lbm_ensemble_sync(lbm_ensemble *ens);
int lbm_ensemble_tune(lbm_ensemble *ens, int32_t knob, int64_t value);
const char *lbm_ensemble_last_error(const lbm_ensemble *ens);
void lbm_ensemble_destroy(lbm_ensemble *ens);

/* lbm_fmap - host precompute of the wall-velocity ratio F of Sec. 2.3 (Eq. F),
 * the ratio of the oscillating axial velocity of elastic-tube Womersley flow
 * (Sec. 2.2) at the displaced wall r = R to that at the fluid node
 * r = R - dr:
 *   F(alpha, dr/R) = (1 - M) / (1 - M J0(Lambda (1 - dr/R)) / J0(Lambda)),
 *   Lambda = i^(3/2) alpha,
 * with the elastic-tube coefficient M = M_re + i M_im supplied by the caller
 * (the paper does not fix it).  out [n_alpha][n_dr][2] host: (Re F, Im F) for
 * every alpha[a] in [0, 25] and dr_over_R[b] in [0, 1); the magnitude |F| is
 * the real ratio a caller passes to lbm_set_wall_params.  A pair whose
 * denominator vanishes (dr = 0 with M = 1) gives NaN.  LBM_EINVAL for
 * arguments out of range.  Runs on the host; no context, no GPU. */
int lbm_fmap(const double *alpha, int64_t n_alpha, const double *dr_over_R, int64_t n_dr,
             double M_re, double M_im, double *out);

/* lbm_tune - launch knobs of one lattice (no effect on results beyond the
 * rounding of the collision arithmetic): LBM_TUNE_PREFETCH (L2 prefetch
 * distance of the bulk kernel, tiles, >= 0), LBM_TUNE_BULK_SITES (1 to 4:
 * one or two sites per lane of the bulk kernel and their pairing) and
 * LBM_TUNE_BULK_WARPS (4 or 8 warps per CTA of the bulk kernel), as for
 * lbm_ensemble_tune, and LBM_TUNE_GRAPH_STEPS: G > 0 (even) replays whole
 * blocks of G steps of lbm_step as one CUDA graph, captured on first use on a
 * stream of the library's own that is ordered with the context's stream by
 * events (the inlet time reads a device step counter; any later lbm_tune or
 * lbm_set_wall_params captures again; not used by lbm_step_diag, while
 * lbm_profile is on, or in checked builds; default 20, 0 for direct
 * launches); for a lattice with 16-bit storage LBM_TUNE_BULK_SITES
 * also takes 5: as 2, but on even steps a fixed grid of warps whose rows
 * arrive by TMA tensor copies into a two-stage shared-memory ring per warp
 * (the first use builds the tensor map of the population array; the same
 * results as 2, bit for bit).  Defaults are chosen per storage at build
 * time.  LBM_EINVAL for another knob or value, LBM_ECUDA when the tensor map
 * cannot be made. */
int lbm_tune(lbm_ctx *ctx, int32_t knob, int64_t value);

/* lbm_set_stream - run subsequent work on another cudaStream_t. */
int lbm_set_stream(lbm_ctx *ctx, void *cuda_stream);

/* lbm_last_error - message of the last failing call on ctx ("" if none),
 * valid until the next call on ctx; with ctx == NULL, the message of the last
 * failed lbm_build_lattice on the calling thread.  lbm_status_string - name of
 * a status. */
const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(int status);

/* lbm_destroy - wait for the stream, free all device and host memory. NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
