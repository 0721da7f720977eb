/*
 * mhd_bunch.h -- C ABI of libmhdbunch.so, the GB300 (sm_103a) MHD bunch update.
 *
 * A *bunch* is a set of patches (small blocks of cells with ghost layers) that are
 * advanced together, one synchronous time step at a time, by the ideal-MHD scheme of
 * Haahr et al. (Sec. 2.1: conservative form Eqs. 1-6, adiabatic EOS; MUSCL-Hancock
 * predictor of Sec. 2.1.4; HLLD face flux of Sec. 2.1.2; constrained transport with an
 * edge EMF from a two-dimensional Riemann solve, Sec. 2.1.3 and Eq. 12).  Patch
 * bunching is Secs. 2.3-2.4 of the paper.
 *
 * State layout (shared by every entry point): the state is ONE device buffer of reals
 * (float when real_bytes == 4, double when 8).  Patch p starts at element
 * patch_offsets[p] (from mhd_bunch_state_size) and is stored as [8][Z][Y][X], x fastest,
 * variables (rho, rho*u, rho*v, rho*w, E, Bx, By, Bz).  Active axes carry `guard` ghost
 * cells on each side; an axis whose box extent is 1 is collapsed and carries none.
 * Bx at local x-index i is the face field on the low x-face of cell i (the index
 * convention of Eqs. 8-12); By, Bz likewise on the low y- and z-faces.
 *
 * Ownership: the caller owns the two state buffers and the CUDA stream (they are only
 * borrowed through mhd_bunch_bind).  The library owns the device patch table, its work
 * buffers, the CUDA graph and the error word, all released by mhd_bunch_destroy.
 *
 * Errors: every function returns an mhd_status (0 on success) and never aborts or throws
 * across the ABI (a failed host allocation inside the library returns MHD_ENOMEM).
 * mhd_last_error() gives a thread-local message for the last failure.
 * Problems found on the device (non-finite or non-positive density / energy after an
 * update, bad patch-table entries, a bounded wait that ran out) are latched in a device
 * error word and reported by the next call that synchronises (mhd_bunch_cfl_dt,
 * mhd_bunch_get_error, mhd_bunch_advance_host).
 *
 * Threading: calls on one handle are stream-ordered on the bound stream and must not be
 * made from several host threads at once.  Different handles are independent.
 */
#ifndef MHD_BUNCH_H
#define MHD_BUNCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mhd_bunch mhd_bunch;

typedef enum {
    MHD_OK = 0,
    MHD_EINVAL = -1,    /* invalid argument (sizes, nvar, guard, null pointer, bad table) */
    MHD_ENOMEM = -2,    /* device or host allocation failed */
    MHD_ECUDA = -3,     /* a CUDA runtime call failed */
    MHD_EPHYS = -4,     /* the device found a non-physical state (rho <= 0, non-finite) */
    MHD_EBOUNDS = -5,   /* the device found an index outside the patch table / buffers */
    MHD_ETIMEOUT = -6,  /* a bounded device wait ran out */
    MHD_ESTATE = -7     /* call out of order (e.g. step before bind / set_geometry) */
} mhd_status;

enum { MHD_BC_PERIODIC = 0, MHD_BC_OUTFLOW = 1 };
enum { MHD_LIMITER_MINMOD = 0, MHD_LIMITER_MC = 1 };
/* Face-flux solver of the update (a7): HLLD (Sec. 2.1.2, the default) or HLL (the simple
 * solver of the paper's mockup, Sec. 2.4).  The edge EMF (a8) is the same for both. */
enum { MHD_RIEMANN_HLLD = 0, MHD_RIEMANN_HLL = 1 };

/* How mhd_bunch_step launches the update kernel.
 *   PER_PATCH  : one launch per patch (the plain path),
 *   BUNCHED    : one launch over every tile of every patch,
 *   PERSISTENT : one launch of (SM count x resident CTAs) CTAs that pull tiles from a
 *                device work counter until the bunch is done,
 *   MIXED      : for bunches of several patch sizes: each patch-size class takes its own
 *                tile configuration (chosen per class by mhd_bunch_autotune) and the
 *                update is one persistent launch per configuration in use, over the
 *                tiles of its patches; until mhd_bunch_autotune has run in this mode, as
 *                PERSISTENT.
 *   BUNCH_LISTS: the paper's bunches (Secs. 2.3-2.4: a bunch of patches per kernel
 *                invocation): one persistent launch per bunch of mhd_bunch_set_bunches,
 *                in list order, over that bunch's tiles; MHD_ESTATE until bunches are set.
 * The streamed and asynchronous advances use the single configuration of
 * mhd_bunch_set_mode in every mode.                                                      */
enum {
    MHD_MODE_PER_PATCH = 0,
    MHD_MODE_BUNCHED = 1,
    MHD_MODE_PERSISTENT = 2,
    MHD_MODE_MIXED = 3,
    MHD_MODE_BUNCH_LISTS = 4
};

/* Create a bunch of npatch equal patches of nx*ny*nz active cells.
 * guard: ghost width on active axes; must be >= 3 (the update reads two ghost cells
 *        plus the far face of the normal field; the paper's patches use 3, Sec. 3.2).
 * nvar : must be 8.  real_bytes: 4 (float) or 8 (double).
 * A dimension of 1 marks a collapsed axis; the active axes must be x, x-y or x-y-z.
 * On success *out holds a new handle.  Returns MHD_EINVAL on bad sizes. */
int mhd_bunch_create(int nx, int ny, int nz, int guard, int nvar, int npatch,
                     int real_bytes, mhd_bunch **out);

/* As mhd_bunch_create, with per-patch sizes: patch_n is host int32[npatch*3]
 * (nx, ny, nz per patch).  The array is copied. */
int mhd_bunch_create_ragged(const int32_t *patch_n, int npatch, int guard, int nvar,
                            int real_bytes, mhd_bunch **out);

/* Place the patches in the box (needed by the guard fill, Sec. 2.2: DISPATCH fills ghost
 * zones from neighbouring patches).
 * dx           host double[3]: cell size along x, y, z.
 * patch_origin host int64[npatch*3]: global cell index of each patch's first active cell.
 * domain_cells host int64[3]: cells of the whole box; extent 1 on collapsed axes.
 * bc           host int32[6]: (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi) boundary kinds,
 *              MHD_BC_PERIODIC or MHD_BC_OUTFLOW (zero-gradient copy).
 * The patches must tile the box exactly (checked; MHD_EINVAL otherwise). */
int mhd_bunch_set_geometry(mhd_bunch *b, const double dx[3], const int64_t *patch_origin,
                           const int64_t domain_cells[3], const int32_t bc[6]);

/* Scheme parameters: adiabatic index, Courant number for mhd_bunch_cfl_dt, slope limiter
 * (MHD_LIMITER_MINMOD or MHD_LIMITER_MC).  Defaults: 5/3, 0.8, minmod. */
int mhd_bunch_set_params(mhd_bunch *b, double gamma, double courant, int limiter);

/* Face-flux solver (MHD_RIEMANN_HLLD or MHD_RIEMANN_HLL) of the step and of its adjoint;
 * default HLLD.  MHD_EINVAL for another value.  Discards a captured graph. */
int mhd_bunch_set_riemann(mhd_bunch *b, int solver);

/* Bytes of one state buffer; if patch_offsets is not NULL it receives npatch int64 element
 * offsets (in reals) of the patches inside the buffer. */
int mhd_bunch_state_size(const mhd_bunch *b, size_t *bytes, int64_t *patch_offsets);

/* Borrow the caller's device buffers (state = current U^n, state_next = where U^{n+1}
 * is written) and CUDA stream (a cudaStream_t, NULL for the legacy default stream).
 * Both buffers must hold mhd_bunch_state_size bytes and be 16-byte aligned. */
int mhd_bunch_bind(mhd_bunch *b, void *state, void *state_next, void *cuda_stream);

/* Device pointer of the buffer that currently holds U^n (the two bound buffers swap
 * roles after every step). */
int mhd_bunch_current(const mhd_bunch *b, void **state);

/* a1: fill every ghost cell of every patch with the box cell it stands for (a copy from
 * the owning patch at the same time, periodic wrap or zero-gradient at the box ends).
 * Stream-ordered, asynchronous. */
int mhd_bunch_fill_guards(mhd_bunch *b);

/* a2: CFL time step dt = courant / max_cells sum_d (|u_d| + c_f,d)/dx_d over the
 * interior cells of all patches (synchronous bunch time step).  Reads the ghost faces
 * next to the interior, so call after mhd_bunch_fill_guards.
 * _device writes the double into dt_dev (device memory) without synchronising;
 * the host variant synchronises the stream and checks the device error word. */
int mhd_bunch_cfl_dt(mhd_bunch *b, double *dt_host);
int mhd_bunch_cfl_dt_device(mhd_bunch *b, void *dt_dev);

/* a1 + a2: the guard fill followed by the CFL dt into dt_dev (device double), as
 * mhd_bunch_fill_guards then mhd_bunch_cfl_dt_device (the same ghost cells and, bitwise,
 * the same dt); for equal patches on a regular grid in one pass over the state (one CTA per
 * padded z-plane fills the plane's ghost cells, then takes the rates of its cells).  The
 * captured graph and the advance calls use it.  Asynchronous, graph-capturable. */
int mhd_bunch_fill_cfl_device(mhd_bunch *b, void *dt_dev);

/* a3-a9: advance every patch by dt: reads U^n (ghosts filled) from the current buffer,
 * writes the interior cells and owned faces of U^{n+1} into the other one, then swaps
 * the two.  Ghost cells of the new state are stale until the next fill. */
int mhd_bunch_step(mhd_bunch *b, double dt);
/* As mhd_bunch_step with dt read on the device from dt_dev (double). */
int mhd_bunch_step_device_dt(mhd_bunch *b, const void *dt_dev);

/* Asynchronous per-patch time stepping (DISPATCH's patches at their own times, Sec. 2.2,
 * updated in bunches of the patches that are ready, Sec. 2.4).  Advances every patch by
 * t_span from the common time of the current state, in rounds.  Each patch keeps two time
 * slices (the current one and the one before; the two bound buffers hold them, patch by
 * patch).  A patch is ready when it is short of t_span and no neighbour (a patch owning a
 * cell of its guard zone) is at an earlier time; every round updates all ready patches as
 * one bunch:  guard zones filled at each patch's own time (the neighbours' two slices
 * interpolated linearly in time), the patch's own CFL dt (courant / max rate over its
 * cells) clipped to what is left of t_span, the update by that dt.  Conservation and
 * div B hold inside patches; faces shared by patches at different times are updated by
 * each side with its own fluxes.  Returns the rounds and the patch updates done; after
 * the call the current buffer holds every patch at the common time + t_span (ghost cells
 * not meaningful).  max_rounds >= 1; MHD_ESTATE if max_rounds ran out first (*rounds and
 * the record still cover the rounds done); MHD_EPHYS if a patch's dt came out
 * non-positive or non-finite (later rounds are skipped; the state is then not meaningful).
 * The schedule runs on the device: each round is five stream-ordered launches (schedule,
 * guard fill at the patches' own times, per-patch CFL dt, dt clipping, update); the host
 * enqueues 32 rounds at a time and synchronises the bound stream once per 32 rounds to
 * read their record. */
int mhd_bunch_advance_async(mhd_bunch *b, double t_span, int max_rounds, int *rounds,
                            int64_t *patch_updates);
/* The record of round `round` of the last mhd_bunch_advance_async: its patches (in
 * ascending order) and the dt each took.  *n receives the count; patches / dts (either may
 * be NULL) must hold cap >= *n entries. */
int mhd_bunch_async_round(const mhd_bunch *b, int round, int32_t *patches, double *dts, int cap,
                          int *n);

/* Bunches of the patches for MHD_MODE_BUNCH_LISTS (Secs. 2.3-2.4: the solver updates a
 * bunch of patches per call; the paper's best bunches hold 100-400 patches).  Bunch q holds
 * patches[starts[q] .. starts[q+1]-1]; starts has nbunch+1 entries, starts[0] = 0 and
 * starts[nbunch] = npatch, and patches lists every patch exactly once (MHD_EINVAL
 * otherwise, nothing changed).  Copied by the library (its tile lists are built here, on
 * the device); a later set_geometry discards them.  After set_geometry (MHD_ESTATE before). */
int mhd_bunch_set_bunches(mhd_bunch *b, const int32_t *patches, const int32_t *starts, int nbunch);

/* Launch mode of the update (MHD_MODE_*) and tile configuration index (0..n-1 from
 * mhd_bunch_num_configs; -1 = library default).  Every mode and every configuration
 * computes bitwise the same state. */
int mhd_bunch_set_mode(mhd_bunch *b, int mode, int config);
int mhd_bunch_num_configs(const mhd_bunch *b, int *nconfig);
int mhd_bunch_config_info(const mhd_bunch *b, int config, int *tile_x, int *tile_y,
                          int *threads);

/* Time each tile configuration on the bound state (a few steps each, the state is
 * restored afterwards) and keep the fastest.  If cache_path is not NULL the choice is
 * read from / written to that text file, keyed by device, precision and patch sizes.
 * In MHD_MODE_MIXED every patch-size class is timed with every configuration on its own
 * tiles and takes its fastest (cache_path is not used); *chosen receives the
 * configuration of the class holding the most cells. */
int mhd_bunch_autotune(mhd_bunch *b, const char *cache_path, int *chosen);

/* Capture nsteps of (fill guards -> CFL dt on the device (mhd_bunch_fill_cfl_device) ->
 * step with the device dt) into
 * a CUDA graph on the bound stream (which must not be the legacy default stream);
 * mhd_bunch_graph_launch replays it and swaps the buffers as the eager steps would.
 * dt_dev (device double[nsteps], may be NULL) receives the dt of each replayed step.
 * Any later set_geometry / set_params / set_mode / bind discards the graph. */
int mhd_bunch_graph_capture(mhd_bunch *b, int nsteps, void *dt_dev);
int mhd_bunch_graph_launch(mhd_bunch *b);

/* End-to-end helper working on HOST memory: copies host_state (state_size bytes, layout
 * above) to the current device buffer, runs nsteps of fill -> CFL dt -> step, copies the
 * final state back into host_state and returns the simulated time advanced in *t_out.
 * Synchronises the bound stream. */
int mhd_bunch_advance_host(mhd_bunch *b, void *host_state, int nsteps, double *t_out);

/* Host-resident state streamed through the GPU every step (bunches staged from the host
 * for each update and returned, Secs. 2.4 and 4 of the paper), with copies overlapped with
 * the update: the state in host_state (state_size bytes, layout above; page-locked memory
 * for the copies to overlap) is cut into at most nchunks contiguous runs of patches (when
 * nchunks equal runs would each hold at least one wave of the persistent update, i.e. SM
 * count x occupancy tiles, the runs are cut at whole waves instead).  Per step:
 * every chunk is copied to the device (on a library-owned stream; chunk k as soon as the
 * previous step returned it), then guard fill -> CFL dt -> the update chunk by chunk on
 * the bound stream, each updated chunk copied back into host_state (on a second library
 * stream) while the next chunk is updated.  After nsteps steps host_state holds the final
 * state (its ghost cells are not meaningful), the device buffer current afterwards holds
 * it too, and *t_out (may be NULL) the simulated time.  nsteps >= 1, 1 <= nchunks (more
 * chunks than patches are capped); the bound stream must not be the legacy default
 * stream.  Synchronises the bound stream; returns the device error word as
 * mhd_bunch_get_error would. */
int mhd_bunch_advance_streamed(mhd_bunch *b, void *host_state, int nsteps, int nchunks, double *t_out);

/* Interior layout: the cells a patch owns, without ghost cells.  Patch p starts at element
 * patch_offsets[p] and is stored as [8][nz][ny][nx], x fastest (variables and face-field
 * convention of the state layout; nx, ny, nz the patch's cells).  *bytes receives the
 * size of the whole interior state; patch_offsets (may be NULL) npatch entries. */
int mhd_bunch_interior_size(const mhd_bunch *b, size_t *bytes, int64_t *patch_offsets);

/* As mhd_bunch_advance_streamed, with the host state in the interior layout
 * (mhd_bunch_interior_size bytes; page-locked for the copies to overlap): ghost cells are
 * derived data (the guard fill rebuilds them before every update), so each step moves
 * only the owned cells, 1/1.675 of the state layout's bytes for 32^3 patches with guard 3.
 * Per step, chunk k is copied into a library-owned device staging buffer (one interior
 * state, allocated on first use, released by mhd_bunch_destroy), scattered into the
 * current state buffer by a copy kernel, and after the update of its patches gathered
 * from the new state into the staging buffer and copied back into host_interior.  The
 * results (host_interior, the device state current afterwards, *t_out) equal those of
 * mhd_bunch_advance_streamed bitwise on the interior.  Same argument rules, errors and
 * synchronisation as mhd_bunch_advance_streamed; MHD_EINVAL as well if a padded patch
 * holds 2^31 or more 4-byte words. */
int mhd_bunch_advance_streamed_interior(mhd_bunch *b, void *host_interior, int nsteps, int nchunks,
                                        double *t_out);

/* ---------------------------------------------------------------------------------------
 * Slabs of a z-layer decomposition of the box (one handle per GPU of a domain split over
 * several GPUs; patches are independent given their guard zones, Secs. 2.2 and 4).
 *
 * mhd_bunch_set_slab, called once after mhd_bunch_set_geometry (the whole box: equal
 * patches on a grid, x fastest, then y, then z, 3D), makes the handle own the patch layers
 * z0 <= layer < z1 only.  Its state (mhd_bunch_state_size, to be bound again with
 * mhd_bunch_bind) then holds the L = z1 - z0 owned layers in slots 0..L-1 and two halo
 * layers: slot L the layer below z0, slot L+1 the layer above z1-1 (periodic wrap across
 * the box; across an outflow box face the halo is never read).  Guard fill, CFL dt, steps,
 * graphs, modes and the autotuner act on the owned patches, reading the halo slots where
 * the guard zones reach the neighbouring layers; the streamed, out-of-core and
 * asynchronous advances and the adjoint are not available (MHD_EINVAL).  Patch p of the
 * handle is owned patch p (layer z0 + p / patches_per_layer), mhd_bunch_interior_size and
 * the interior layout refer to the owned patches.
 *
 * Per step the caller exchanges halos: mhd_bunch_slab_pack copies the interiors of the
 * bottom and top owned layers of the current state into `bottom` / `top` (device buffers
 * of layer_bytes, interior layout of one layer's patches in order; either may be NULL);
 * the neighbours' copies arrive through the caller's transport (NCCL, peer copies, ...)
 * and mhd_bunch_slab_unpack writes them into the halo slots of the current state (below:
 * the top layer of the slab underneath, above: the bottom layer of the slab on top; either
 * may be NULL).  Then guard fill + dt on the slab, the minimum dt over all slabs, and the
 * step.  Stream-ordered on the bound stream.  MHD_ESTATE before set_geometry, on a handle
 * that is a slab already (set_slab) or is not one (info, pack, unpack); MHD_EINVAL for other
 * geometries (or more than 65535 patches per z-layer) or layer ranges. */
int mhd_bunch_set_slab(mhd_bunch *b, int z0, int z1);
int mhd_bunch_slab_info(const mhd_bunch *b, int *layers, int64_t *patches_per_layer,
                        size_t *layer_bytes);
int mhd_bunch_slab_pack(mhd_bunch *b, void *bottom, void *top);
int mhd_bunch_slab_unpack(mhd_bunch *b, const void *below, const void *above);

/* Host-resident state larger than the device memory this call may use (the paper's
 * bunches staged from the host every update, Secs. 2.4 and 4, for a domain that does not
 * fit in HBM).  host_state holds the state in the interior layout (mhd_bunch_interior_size
 * bytes; page-locked for the copies to overlap); host_scratch is a second buffer of the
 * same size (different from host_state) that the call writes freely.  After nsteps steps
 * host_state holds the new state and *t_out (may be NULL) the simulated time.
 *
 * Only for a 3D box of equal patches on a grid, listed x fastest, then y, then z (as
 * mhd_bunch_create makes them); its z-layers of patches are the unit of transfer.  The
 * call allocates at most device_budget bytes of device memory for its working set (the
 * handle's own tables, allocated earlier, come on top; bind is not needed): a ring of
 * L+2 padded layers for U^n and one for U^{n+1}, upload and download stages and tables,
 * with L the largest chunk of layers that fits (MHD_ENOMEM if one layer does not).  Per
 * step, two passes over the chunks, each window of layers uploaded once per pass, its
 * layers above and below included: (1) guard fill + CFL rates of every chunk, dt = the
 * smallest chunk dt, i.e. the global CFL dt; (2) guard fill and update of each chunk, in
 * reverse order (the last chunk's window is still on the device), its new interior copied
 * back into the other host buffer.  The results equal those of
 * the device-resident steps (mhd_bunch_fill_cfl_device + mhd_bunch_step_device_dt)
 * bitwise.  Runs on cuda_stream (NULL: legacy default stream) and the library's copy
 * streams and synchronises them; returns the device error word as mhd_bunch_get_error
 * would.  io_bytes (may be NULL) receives the bytes copied host -> device and device ->
 * host over the call.  MHD_EINVAL for other geometries (or more than 65535 patches per z-layer) or bad
 * arguments, MHD_ESTATE before set_geometry. */
int mhd_bunch_advance_out_of_core(mhd_bunch *b, void *host_state, void *host_scratch, int nsteps,
                                  size_t device_budget, void *cuda_stream, double *t_out,
                                  size_t io_bytes[2]);

/* Adjoint of one step at fixed dt (the reverse of mhd_bunch_step, including the guard
 * fill): given U^n (interior valid; ghosts are re-filled internally) and the cotangent
 * lam_next of U^{n+1} (interior cells and owned faces), writes
 * lam = (dU^{n+1}/dU^n)^T lam_next on the interior cells and owned faces, summing the
 * contributions that reached ghost copies back into the cells they copy.  All three are
 * device buffers in the state layout; lam is overwritten.  Ghost entries of lam_next are
 * ignored and those of lam are set to 0.  Non-differentiable points take the subgradient
 * of the forward branch (limiter: the selected argument, zero when the arguments differ
 * in sign; wave-speed max/min: the selected argument, first on ties). */
int mhd_bunch_step_adjoint(mhd_bunch *b, double dt, const void *U_n, const void *lam_next,
                           void *lam);

/* Device error word: *code receives the latched mhd_status (MHD_OK if none) and msg (if
 * not NULL) a description; the word is cleared.  Synchronises the stream. */
int mhd_bunch_get_error(mhd_bunch *b, int *code, char *msg, size_t len);

/* Number of the library's own kernel launches issued on this handle so far. */
int mhd_bunch_launch_count(const mhd_bunch *b, int64_t *count);

void mhd_bunch_destroy(mhd_bunch *b);

/* Thread-local text of the last error returned by any call on this thread. */
const char *mhd_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Allocation-free CFL time step.  The paper has no counterpart: this entry point exists
 * for callers that must not allocate device memory through the CUDA runtime -- hosts whose
 * framework hands out all device memory from its own pool and accounts for every byte,
 * real-time loops that cannot afford an allocation.  It needs no handle and calls no
 * cudaMalloc / cudaFree (nor any other allocating routine): its scratch is a static device
 * array inside the library holding one partial maximum per patch, MHD_NOALLOC_MAX_PATCHES
 * entries (128 KB of doubles plus a 4-byte counter), which every GPU that loads the
 * library keeps until the process exits.
 *
 * Computes the same dt as mhd_bunch_cfl_dt (courant / max over interior cells of
 * sum_d (|u_d| + c_f,d)/dx_d) for `npatch` equal patches of nx*ny*nz active cells stored
 * back to back in the state layout above (patch p at element p*8*X*Y*Z, guard ghosts on
 * active axes; ghost faces next to the interior must be filled).  Writes the double dt
 * to dt_dev (device memory) on cuda_stream (NULL: legacy default stream) without
 * synchronising.  real_bytes 4 or 8; npatch above MHD_NOALLOC_MAX_PATCHES is rejected
 * with MHD_EINVAL before any device work.  A cell whose rate is not finite (non-physical
 * state) makes the written dt NaN, so that a caller stepping with dt_dev on the device
 * carries the failure forward instead of stepping with a dt that ignores the cell.
 *
 * cuda_stream must belong to the current device (MHD_EINVAL otherwise).  Every call shares
 * the one static array, which keeps the last call's contents (the counter that must start
 * at zero is cleared on the stream before each launch): calls whose kernels may overlap on
 * the GPU, e.g. on two streams at once, race and must be ordered by the caller.  The first
 * call on a device looks up the array's device address (with that device current; a
 * lookup that fails is retried by the next call); make that first call before any stream
 * capture begins.  A CUDA error already pending on the calling thread when the call starts
 * is cleared, so that MHD_ECUDA reports this call's own failure. */
#define MHD_NOALLOC_MAX_PATCHES 16384
int mhd_cfl_dt_uniform_noalloc(const void *state, int real_bytes, int npatch, int nx, int ny,
                               int nz, int guard, const double dx[3], double gamma,
                               double courant, void *dt_dev, void *cuda_stream);

/* Attainable SIMT fused multiply-add rate of the current device, the denominator of the
 * arithmetic roofline of the fused step (which has no dense contraction and runs on the
 * FP32 / FP64 SIMT pipes, not on the tensor cores).  Runs independent FMA chains on four
 * 256-thread blocks per SM on cuda_stream (NULL: legacy default stream), one warm-up and
 * three timed launches, synchronising the stream; writes the best rate, counting 2 flops
 * per FMA, to *flops_per_second.  real_bytes 4 (FP32) or 8 (FP64).  Takes tens of
 * milliseconds (FP32) and allocates nothing.  MHD_EINVAL for a bad argument (checked
 * before any device call), MHD_ECUDA for a CUDA error. */
int mhd_probe_fma_rate(int real_bytes, void *cuda_stream, double *flops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* MHD_BUNCH_H */
