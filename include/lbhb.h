/*
 * lbhb: GB300 (sm_103a) library for the two-species lattice Boltzmann model
 * with multirange Shan-Chen interactions of Benzi, Bernaschi, Sbragaglia and
 * Succi, "Herschel-Bulkley rheology from lattice kinetic theory of soft-glassy
 * materials" (arXiv 1004.5058).
 *
 * Model (section "Lattice Boltzmann with multirange interactions"):
 *   Eq. (be)  f_is(r+c_i,t+1) - f_is(r,t) = -(1/tau)[f_is - f^eq_is(rho_s, u + tau F_s/rho_s)],
 *             s = A,B, D2Q9 populations, f^eq second order in u, cs^2 = 1/3;
 *   Eq. (FFF) F_s = F^a_s + F^r_s + F^X_s: attractive belt-1 self force, repulsive
 *             two-belt (24 neighbours) self force, belt-1 cross-species repulsion,
 *             on the pseudopotential psi(rho) = rho0 (1 - exp(-rho/rho0)).
 * One relaxation time tau for both species, as in all the paper's runs, unless
 * a cell sets tau_b (a time per species; see lb_cell_params).
 * Boundaries: periodic in x; in y periodic or Couette (halfway bounce-back walls
 * at y = -1/2 and y = ny - 1/2 moving at -u_wall and +u_wall in x; the paper
 * itself uses a fully periodic box, walls are an extension for shear-rate control).
 *
 * Conventions for every call:
 *  - the return value is an lb_status; LB_OK = 0 on success;
 *  - arrays the caller passes are caller-owned; the library copies what it needs
 *    and never keeps or frees a caller pointer;
 *  - host field arrays are float64, laid out [cell][y][x] with x fastest;
 *  - one handle is used by one host thread at a time;
 *  - work is enqueued on the handle's CUDA stream (the caller's stream given at
 *    lb_create, or a library-owned stream); calls that return data to the host
 *    synchronise that stream;
 *  - errors found on the device (non-finite or non-positive density) are
 *    reported by the next call that synchronises, as LB_ERR_NONFINITE; the handle
 *    then refuses lb_step with LB_ERR_STATE until lb_init_fields or
 *    lb_set_populations loads a new state;
 *  - lb_last_error returns a message for the last failing call of a handle.
 */
#ifndef LBHB_H
#define LBHB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle; /* opaque; created and freed by the library */

typedef enum {
    LB_OK = 0,
    LB_ERR_INVALID = -1,     /* bad argument (null pointer, size, tau <= 1/2 ...) */
    LB_ERR_CUDA = -2,        /* a CUDA runtime/driver call failed */
    LB_ERR_NOMEM = -3,       /* device or host allocation failed */
    LB_ERR_NONFINITE = -4,   /* the device found a non-finite or non-positive density */
    LB_ERR_TIMEOUT = -5,     /* a bounded device wait ran out */
    LB_ERR_STATE = -6,       /* call not valid in the handle's current state */
    LB_ERR_UNSUPPORTED = -7  /* valid request this build or shape does not support */
} lb_status;

typedef enum { LB_BC_PERIODIC = 0, LB_BC_COUETTE = 1 } lb_bc;

/* Storage precision of the populations.  Arithmetic is FP32 for LB_FP32 and
 * LB_FP16_SHIFTED (populations stored as g_i = f_i - w_i rho_bar_s in FP16,
 * round to nearest) and FP64 for LB_FP64.  LB_FP16_SHIFTED_SR stores 4096 g_i
 * in FP16 with stochastic rounding in the time step (unbiased: the stored value
 * equals the computed one in expectation, so rounding errors do not accumulate
 * into a drift of mass or momentum in near-uniform states); the random bits come
 * from a hash of each site and its densities, so runs are reproducible.  Its
 * 2 bytes per value and FP32 arithmetic are those of LB_FP16_SHIFTED.  The paper
 * stores populations in one precision and says nothing of reduced storage.
 * Observables are reduced in FP64. */
typedef enum { LB_FP32 = 0, LB_FP16_SHIFTED = 1, LB_FP64 = 2, LB_FP16_SHIFTED_SR = 3 } lb_precision;

/* Kernel family: AUTO picks TILED when the shape allows it, else GENERIC. */
typedef enum { LB_KERNEL_AUTO = 0, LB_KERNEL_GENERIC = 1, LB_KERNEL_TILED = 2 } lb_kernel;

/* One lattice cell, in the paper's symbols.  All cells of a handle share nx, ny
 * and bc; the other fields may differ per cell (batched flow curves).
 *   tau      BGK relaxation time (Eq. (be)) of both species, or of species A
 *            when tau_b is set; must be > 1/2
 *   rho0     reference density of psi(rho) = rho0 (1 - exp(-rho/rho0)) and of F^X
 *   g_aa1, g_bb1  G^a_AA, G^a_BB: belt-1 self couplings (negative attracts)
 *   g_aa2, g_bb2  G^r_AA, G^r_BB: two-belt self couplings (positive repels)
 *   g_ab     G_AB = G_BA: belt-1 cross-species coupling
 *   u_wall   Couette wall speed U (bottom wall -U, top wall +U); ignored if periodic
 *   f0       amplitude of the Kolmogorov body force F_x(y) = f0 sin(2 pi y / ny) of
 *            section "Numerical Results" (force density; each species receives
 *            rho_s / rho of it); 0 for none
 *   rho_bar_a, rho_bar_b  shift reference of LB_FP16_SHIFTED storage
 *   bc       lb_bc
 *   tau_b    relaxation time of species B (> 1/2), or 0 for tau.  The paper runs
 *            one time for both species (tau = 1) and names a coupling-dependent
 *            one as unexplored (footnote of section "Numerical Results").  With
 *            tau_b != tau, tau is species A's, each species relaxes with its own
 *            time and is shifted by tau_s F_s / rho_s, and u in Eq. (be) is the
 *            common velocity (j_A/tau_A + j_B/tau_B) / (rho_A/tau_A + rho_B/tau_B)
 *            of Shan and Doolen (J. Stat. Phys. 81, 1995), which keeps the
 *            collision from creating momentum; tau_b = tau gives the one-time
 *            model bit for bit.
 *   s_e, s_eps, s_q, s_nu  rates of a multiple-relaxation-time collision, each
 *            in (0, 2), or 0 for 1/tau_s (a method variant, not in the paper;
 *            the same footnote's unexplored relaxation).  The collision becomes
 *            f* = f - M^-1 S M (f - f^eq) on the orthogonal D2Q9 moments of
 *            Lallemand and Luo (Phys. Rev. E 61, 2000): density and momentum
 *            relax with 1/tau_s (so tau_s still sets the force shift tau_s F_s /
 *            rho_s), the energy e with s_e, its square eps with s_eps, the energy
 *            fluxes q_x, q_y with s_q and the stresses p_xx, p_xy with s_nu,
 *            which sets the shear viscosity (1/s_nu - 1/2)/3.  With all four 0
 *            the collision is the paper's BGK one.  A batch in which any cell
 *            sets a rate runs every cell through the MRT update (cells without
 *            rates then get the BGK result to rounding, not bit for bit).
 * The fields after bc are last, so callers that fill the fields before them and
 * zero the rest get the paper's model. */
typedef struct {
    int nx, ny;
    double tau, rho0;
    double g_aa1, g_aa2, g_bb1, g_bb2, g_ab;
    double u_wall;
    double f0;
    double rho_bar_a, rho_bar_b;
    int bc;
    double tau_b;
    double s_e, s_eps, s_q, s_nu;
} lb_cell_params;

/* Creates a handle for n_cells cells (n_cells >= 1; nx >= 5, ny >= 5; same nx, ny,
 * bc in every cell) and allocates all device memory it needs.  cuda_stream:
 * a cudaStream_t of the current device, or NULL for a library-owned stream.
 * The populations start undefined: call lb_init_fields or lb_set_populations.
 * Errors: LB_ERR_INVALID, LB_ERR_NOMEM, LB_ERR_CUDA; *out is NULL on failure. */
lb_status lb_create(const lb_cell_params* cells, int n_cells, lb_precision prec,
                    void* cuda_stream, lb_handle** out);

/* Sets f_is = f^eq_is(rho_s, u) (moments and f^eq of Eq. (be)) at every site.
 * rho_a, rho_b: host [n_cells][ny][nx] (required); ux, uy: same shape or NULL
 * for zero.  Resets the step counter to 0, the time averages and the error
 * state.  Synchronous. */
lb_status lb_init_fields(lb_handle* h, const double* rho_a, const double* rho_b,
                         const double* ux, const double* uy);

/* lb_init_fields in two halves, so that the host-to-device copy of the next
 * run's fields overlaps the time steps of the current one (serving many runs
 * of one handle back to back; the paper has no counterpart).
 * lb_stage_fields copies the fields (layout and NULL rules of lb_init_fields)
 * into the handle's staging buffer on a copy stream of its own and returns
 * without waiting; the copy starts once the previous lb_init_fields_staged has
 * read the buffer, and runs beside whatever the handle's stream is doing.  The
 * host arrays must stay valid and unchanged until the lb_init_fields_staged
 * that consumes them returns; with page-locked host memory the copy is
 * asynchronous (pageable memory is copied through a driver bounce buffer and
 * may make the call wait).  A second lb_stage_fields before
 * lb_init_fields_staged replaces the staged fields; lb_init_fields discards
 * them.  The first call allocates the staging buffer.
 * lb_init_fields_staged waits on the host for the staged copy, then enqueues
 * f = f^eq of the staged fields on the handle's stream and returns without
 * synchronising; counters and time averages reset as in lb_init_fields.
 * Errors: LB_ERR_INVALID (rho_a or rho_b NULL), LB_ERR_STATE (nothing staged),
 * LB_ERR_NOMEM, LB_ERR_CUDA. */
lb_status lb_stage_fields(lb_handle* h, const double* rho_a, const double* rho_b,
                          const double* ux, const double* uy);
lb_status lb_init_fields_staged(lb_handle* h);

/* Loads populations from host memory: f [n_cells][2][9][ny][nx] float64
 * (species A then B, D2Q9 order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1)
 * 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)).  Rounded to the storage precision.
 * Resets counters like lb_init_fields.  Synchronous. */
lb_status lb_set_populations(lb_handle* h, const double* f);

/* Copies the populations to host memory in the layout of lb_set_populations
 * (FP16-shifted storage is returned as f = g + w_i rho_bar_s).  Synchronous. */
lb_status lb_get_populations(lb_handle* h, double* f);

/* Advances every cell by n_steps time steps of Eq. (be) (n_steps >= 0).
 * Asynchronous on the handle's stream; returns after enqueueing.  Reports a
 * device error of an earlier, already finished batch if one was recorded. */
lb_status lb_step(lb_handle* h, long long n_steps);

/* Time-averaging window of the shear observables: step t (counted from the
 * last init) is sampled if every > 0, t >= start_step and
 * (t - start_step) % every == 0.  every = 0 disables sampling.  Clears the
 * accumulated averages. */
lb_status lb_set_sampling(lb_handle* h, long long start_step, long long every);

/* Per-cell time averages over the sampled steps (host outputs [n_cells]):
 *   sigma_xy  = (Pi_top - Pi_bot) / (2 nx n_samples), Pi_wall being the x-momentum
 *               the wall delivers to the fluid through bounce-back in one step;
 *   shear_rate = (Ubar(ny-1) - Ubar(0)) / (ny-1), Ubar(y) the time average of the
 *               line average over x of u_x = (j_x + (F_Ax + F_Bx)/2)/rho (the
 *               paper's U_x(y) of section "Numerical Results", force-corrected);
 *   shear_bulk (nullable) = least-squares slope of Ubar over rows [ny/4, ny-ny/4).
 * NaN where no step was sampled.  Synchronous. */
lb_status lb_shear_stress(lb_handle* h, double* sigma_xy, double* shear_rate,
                          double* shear_bulk);

/* Time-averaged line profile Ubar(y), host [n_cells][ny]; number of samples in
 * *n_samples (nullable).  Synchronous. */
lb_status lb_get_profile(lb_handle* h, double* ubar, long long* n_samples);

/* Current fields (host [n_cells][ny][nx], any pointer may be NULL):
 * rho_s = sum_i f_is and the paper's barycentric u = sum_s sum_i f_is c_i / rho
 * (also for cells whose species relax with times of their own).
 * Synchronous; reports LB_ERR_NONFINITE if any density is not finite or <= 0. */
lb_status lb_get_fields(lb_handle* h, double* rho_a, double* rho_b, double* ux, double* uy);

/* FP64 reductions of the current state on the device (host outputs):
 * mass_ab [n_cells][2] = sum of rho_A, rho_B; momentum_xy [n_cells][2] = sum of
 * j_x, j_y.  Either may be NULL.  Synchronous; reports LB_ERR_NONFINITE. */
lb_status lb_reductions(lb_handle* h, double* mass_ab, double* momentum_xy);

/* Chooses the kernel family and tile for subsequent steps.  Tiled family:
 * tile_x = columns per work item (32, 64, 128 or 256, dividing nx; 0 = the
 * widest that divides nx), tile_y = rows per work item (0 = chosen from a
 * model of how evenly the work items fill the GPU).  The generic family
 * ignores both.  LB_ERR_UNSUPPORTED if the shape does not allow the request. */
lb_status lb_set_kernel(lb_handle* h, lb_kernel kernel, int tile_x, int tile_y);

/* Times the supported tiles on this handle's buffers (the state is left
 * unchanged) and selects the fastest.  cache_path (nullable): a text file where
 * results are looked up and stored, keyed by device, shape, cell count and
 * precision.  Synchronous. */
lb_status lb_autotune(lb_handle* h, const char* cache_path);

/* Reads the kernel family and tile in use (outputs nullable). */
lb_status lb_get_kernel(const lb_handle* h, lb_kernel* kernel, int* tile_x, int* tile_y);

/* Launch shape of the tiled kernel in use (outputs nullable): persistent CTAs of
 * plain and of sampled steps (each as many as fit on the GPU, at most one per
 * work item), threads and dynamic shared memory bytes per CTA.
 * LB_ERR_UNSUPPORTED for the generic kernel. */
lb_status lb_launch_shape(const lb_handle* h, int* ctas, int* ctas_sampled, int* threads, int* smem_bytes);

/* Waits for all enqueued work of the handle; reports device errors. */
lb_status lb_sync(lb_handle* h);

/* Number of time steps taken since the last init (0 for NULL). */
long long lb_steps_done(const lb_handle* h);

/* Checkpoint and resume of a long run (the paper's runs take 10^6 steps; it
 * says nothing about restarting them).  lb_save writes the whole state of the
 * handle to the file `path`: the populations in their storage precision (bit
 * for bit), the time step, the sampling window with its time sums, and the cell
 * parameters.  It waits for the handle's work and fails with the pending device
 * error if there is one (LB_ERR_NONFINITE / LB_ERR_TIMEOUT), LB_ERR_STATE if no
 * state is loaded, LB_ERR_INVALID if the file cannot be written.
 * lb_load restores such a file into a handle created with the same number of
 * cells, lattice size, boundary kind and precision (else LB_ERR_INVALID; the
 * cell parameters are taken from the file); a run continued after lb_load
 * equals the run continued after lb_save bit for bit.  A file that is not a
 * checkpoint, is truncated or fails its checksum gives LB_ERR_INVALID and
 * leaves the handle without a loaded state.  Both calls are synchronous; the
 * file is binary in this machine's byte order (format version 2: a 128-byte
 * header, 15 float64 per cell, the float64 time sums, then the populations
 * [cell][s][i][y][x] without row padding, FNV-1a 64 checksum of the payload in
 * the header).  lb_load also reads version 1 files (14 float64 per cell, no
 * tau_b: one relaxation time). */
lb_status lb_save(lb_handle* h, const char* path);
lb_status lb_load(lb_handle* h, const char* path);

/* Test hook for the failure paths (the paper has no counterpart): arms one
 * fault for the next lb_step of this handle.
 *   fault = 1  the first launch of that step leaves one row copy of its first
 *              CTA unissued (tiled kernel only, else LB_ERR_UNSUPPORTED): the
 *              waits for it run out after their 1.5 s bound, the kernel records
 *              a timeout and returns, later launches of the batch exit at once,
 *              and the next synchronising call reports LB_ERR_TIMEOUT.  Nothing
 *              faults: the device stays usable and lb_init_fields recovers.
 *   fault = 2  the step fails at once with LB_ERR_CUDA, as a failed launch
 *              would, without enqueuing anything; the state is unchanged.
 *   fault = 0  disarms.  Other values: LB_ERR_INVALID. */
lb_status lb_test_inject(lb_handle* h, int fault);

/* The cudaStream_t the handle enqueues on (the caller's, or the library's own
 * non-blocking stream), for recording events around lb_step. */
void* lb_stream(const lb_handle* h);

/* Number of CUDA kernel launches the handle has enqueued since creation
 * (kernels launched as nodes of a CUDA graph count one each). */
long long lb_kernel_launches(const lb_handle* h);

/* FP64 state sums without any allocation, for callers that cannot allocate
 * device memory (their memory belongs to another allocator or a fixed budget,
 * or they cannot accept the device-wide synchronisation cudaMalloc/cudaFree
 * may cause).  The paper has no counterpart: it is an interface variant of
 * lb_reductions that needs no handle.
 *   populations  caller's device buffer, layout [n_cells][18][ny][pitch]
 *                (species A then B, D2Q9 order as in lb_set_populations), in
 *                LB_FP32 or LB_FP64 storage; LB_FP16_SHIFTED and
 *                LB_FP16_SHIFTED_SR are rejected (LB_ERR_UNSUPPORTED)
 *   sums         caller's device buffer [n_cells][4] float64, receives
 *                (sum rho_A, sum rho_B, sum j_x, sum j_y) per cell; a
 *                non-finite density makes its cell's sums non-finite.  Unlike
 *                lb_reductions, this variant does not report a non-positive
 *                density (it returns before the work is done): check the sums
 *   cuda_stream  stream of the current device (NULL: the legacy default stream)
 * Before anything is enqueued both buffers are checked: each must be device
 * (or managed) memory of the current device whose allocation holds the bytes
 * the layout needs from the given pointer on (n_cells*18*ny*pitch elements;
 * n_cells*4 doubles), else LB_ERR_INVALID; host memory, another device's
 * memory and too small buffers are refused this way.
 * Work is enqueued and the call returns; read sums after the stream is done.
 * The partial sums live in one scratch array compiled into the library
 * (65536 doubles + an error word, 512 KiB on every GPU that loads the library,
 * held until exit).  A cell needs 4 * min(1024, ceil(nx*ny / 8192)) partial
 * sums, and all cells together at most 65536, else LB_ERR_INVALID with a
 * message: e.g. 16 cells of 4096x4096 fit, 17 do not.  The array is shared by
 * all calls on a device and keeps the last call's contents; calls that overlap
 * on the GPU (different streams or host threads) race on it and must be
 * serialised by the caller.  Every call looks up the array's device address on
 * the current device (cudaGetSymbolAddress); the first call on a device may
 * load the library's device code, so make it before any stream capture.
 * Allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 * Errors: LB_ERR_INVALID (null, misaligned, host or too small buffer, bad
 * size), LB_ERR_UNSUPPORTED, LB_ERR_CUDA; message in lb_last_error(NULL). */
lb_status lb_reductions_noalloc(const void* populations, lb_precision prec, int nx, int ny, int pitch,
                                int n_cells, double* sums, void* cuda_stream);

/* ---- One cell split into horizontal slabs (one handle, and possibly one GPU,
 * per slab).  The paper runs single 512 x 512 lattices for 10^6 steps; larger
 * cells than one GPU holds are split along y.  A slab owns rows [y0, y0 + rows)
 * of each cell and keeps two ghost rows on each side: the interaction stencil of
 * Eq. (FFF) reaches two rows out, and push streaming moves populations one row.
 * Per time step the slabs trade two kinds of rows with their neighbours (the
 * slab below holds the rows just below y0; in a periodic cell the first and last
 * slabs are neighbours; across a Couette wall there is none):
 *   before the step  each slab's first two and last two own rows, all 18
 *                    populations, into the neighbours' ghost rows
 *                    (lb_slab_get EDGE_LO / EDGE_HI, lb_slab_put EDGE_HI / EDGE_LO);
 *   lb_step(h, 1)    the slab's own rows, exactly as the whole-cell step updates
 *                    them, except the populations that stream in from the
 *                    neighbours; those that stream out land in the ghost rows;
 *   after the step   the c_y = -1 populations that left through the lower edge
 *                    into the slab below's last row, the c_y = +1 ones that left
 *                    through the upper edge into the slab above's first row
 *                    (lb_slab_get FLOW_LO / FLOW_HI, lb_slab_put FLOW_HI / FLOW_LO).
 * Done this way, the slabs' rows equal the whole-cell run's bit for bit. */
typedef enum {
    LB_SLAB_EDGE_LO = 0,  /* get: own rows 0, 1; put: the ghost rows below (the slab below's EDGE_HI) */
    LB_SLAB_EDGE_HI = 1,  /* get: own rows rows-2, rows-1; put: the ghost rows above (the slab above's EDGE_LO) */
    LB_SLAB_FLOW_LO = 2,  /* get: the c_y = -1 populations that left downwards; put: the c_y = +1 populations
                             that came up into own row 0 (the slab below's FLOW_HI) */
    LB_SLAB_FLOW_HI = 3   /* get: the c_y = +1 populations that left upwards; put: the c_y = -1 populations
                             that came down into the last own row (the slab above's FLOW_LO) */
} lb_slab_part;

/* Creates a slab handle: rows [y0, y0 + rows) of each of the n_cells cells
 * (cells[].ny is the whole cell's height; rows >= 2; y0 + rows <= ny; a
 * periodic cell needs rows + 4 <= ny).  Like lb_create otherwise; the tiled
 * kernel only (LB_ERR_UNSUPPORTED where its shape rules exclude the cell).
 * On a slab handle every call that takes or returns fields, populations,
 * profiles or sums works on the own rows ([n_cells][rows][nx] host arrays,
 * [n_cells][2][9][rows][nx] populations); lb_step takes one step per call
 * (n_steps 0 or 1, else LB_ERR_INVALID); lb_shear_stress, lb_save and lb_load
 * give LB_ERR_UNSUPPORTED (the stress needs both walls: combine lb_get_profile
 * and lb_wall_momentum over the slabs).  The ghost rows hold nothing until the
 * first exchange: trade edges before the first step. */
lb_status lb_create_slab(const lb_cell_params* cells, int n_cells, lb_precision prec, int y0, int rows,
                         void* cuda_stream, lb_handle** out);

/* First own row, own rows and the whole cell's height of a slab (outputs
 * nullable; for a whole-cell handle 0, ny, ny and LB_ERR_UNSUPPORTED). */
lb_status lb_slab_info(const lb_handle* h, int* y0, int* rows, int* ny_global);

/* Size of a slab message, the same for get and put of a part:
 * EDGE n_cells * 18 * 2 * nx elements, FLOW n_cells * 6 * nx elements, in the
 * storage precision (2, 4 or 8 bytes).  Layout [cell][population][row][x], x
 * dense; FLOW populations in the order 2, 5, 6 (or 4, 7, 8) of species A, then
 * B. */
lb_status lb_slab_message_bytes(const lb_handle* h, lb_slab_part part, size_t* bytes);

/* Packs a message from the slab's current state into the caller's device buffer
 * dst (lb_slab_get), or unpacks one into it (lb_slab_put), on the handle's
 * stream; asynchronous, the copy is ordered with the handle's other work only.
 * The buffer must be device memory of the handle's device holding
 * lb_slab_message_bytes from the pointer on (else LB_ERR_INVALID before
 * anything is enqueued).  Ownership stays with the caller; across devices the
 * caller moves messages between buffers (peer copies, NCCL send/recv).
 * LB_ERR_UNSUPPORTED on a whole-cell handle, LB_ERR_STATE before a state is
 * loaded. */
lb_status lb_slab_get(lb_handle* h, lb_slab_part part, void* dst);
lb_status lb_slab_put(lb_handle* h, lb_slab_part part, const void* src);

/* Time sums over the sampled steps of the x-momentum the walls delivered
 * (sums [n_cells][2] = Pi_top, Pi_bot as in lb_shear_stress, zero for a wall a
 * slab does not hold) and the number of sampled steps (nullable).
 * Synchronous. */
lb_status lb_wall_momentum(lb_handle* h, double* sums, long long* n_samples);

/* Message for the last failing call on h; a static string when h is NULL. */
const char* lb_last_error(const lb_handle* h);

/* Frees the handle and all its device memory.  NULL is a no-op. */
void lb_destroy(lb_handle* h);

/* Herschel-Bulkley fit sigma = sigma_Y + A S^beta (the law the paper fits in
 * section "Numerical Results", written there as A + B S^beta) by variable
 * projection: for each beta the best (sigma_Y, A) is a linear least-squares
 * problem; beta minimises the residual, found by a scan over [beta_lo, beta_hi]
 * and a golden-section refinement.  Host FP64.  Needs n >= 3 points with S > 0.
 * out[0] = sigma_Y, out[1] = A, out[2] = beta, out[3] = residual sum of squares. */
lb_status lb_hb_fit(const double* shear_rate, const double* sigma, int n,
                    double beta_lo, double beta_hi, double* out);

#ifdef __cplusplus
}
#endif
#endif /* LBHB_H */
