/*
 * tersoff.h -- C ABI of the GB300 Tersoff library (libtersoff_gb300.so).
 *
 * The library evaluates the Tersoff multi-body potential (Hoehnerbach, Ismail,
 * Bientinesi, "The Vectorization of the Tersoff Multi-Body Potential", SC'16;
 * Sec. III, Eq. 5-7) -- energy, forces and virial over a neighbour list --
 * and runs velocity-Verlet molecular dynamics with it, on one GPU.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless a comment
 *    says "host". Positions, velocities and forces are row-major N x 3 double
 *    (atom-major, x y z). Species are int32 in [0, n_species).
 *  - Units are "metal": Angstrom, eV, ps, amu.
 *  - The box is orthorhombic and periodic in all three directions, with edges
 *    box[0..2] (host array). Distances use the minimum image convention.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is enqueued on it; an entry point returns after enqueueing
 *    unless its comment says it synchronises the stream.
 *  - Every entry point returns a status code (TERSOFF_OK or TERSOFF_E_*);
 *    tersoff_last_error() gives a one-line description of the last failure on
 *    that context. A failed call leaves caller-owned outputs undefined.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - The entry points that enqueue work (builds, evaluations, backward, MD,
 *    autotuning, halo packing, checkpoints; not tersoff_compute_noalloc) mark
 *    their host call with an NVTX range named after the entry point, which
 *    profilers that record NVTX show around the call's kernels.
 */
#ifndef TERSOFF_GB300_H
#define TERSOFF_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tersoff_ctx tersoff_ctx;

/* status codes */
#define TERSOFF_OK 0
#define TERSOFF_E_INVALID_ARG 1    /* bad pointer, size or value */
#define TERSOFF_E_BOX_TOO_SMALL 2  /* a box edge is shorter than 2 x list radius */
#define TERSOFF_E_NEIGH_OVERFLOW 3 /* neighbour capacity exceeded (see tersoff_neighbor_capacity) */
#define TERSOFF_E_NONFINITE 4      /* non-finite position found while building lists */
#define TERSOFF_E_TIMEOUT 5        /* a bounded device-side wait gave up */
#define TERSOFF_E_CUDA 6           /* a CUDA runtime call failed */
#define TERSOFF_E_STATE 7          /* call out of order (e.g. compute before params) */

/* arithmetic paths */
#define TERSOFF_FP64 0  /* all arithmetic in double (the paper's Opt-D mode, Sec. V-E) */
#define TERSOFF_MIXED 1 /* per-term arithmetic and each atom's own sums over its
                           terms in float; every sum across atoms in double, or in
                           compensated float carried exactly into double (the
                           paper's Opt-M mode, Sec. V-E) */

/* Number of doubles per parameter record and their order. */
#define TERSOFF_NPARAM 14
/* field order inside a record */
#define TERSOFF_P_M 0
#define TERSOFF_P_GAMMA 1
#define TERSOFF_P_LAMBDA3 2
#define TERSOFF_P_C 3
#define TERSOFF_P_D 4
#define TERSOFF_P_H 5
#define TERSOFF_P_N 6
#define TERSOFF_P_BETA 7
#define TERSOFF_P_LAMBDA2 8
#define TERSOFF_P_B 9
#define TERSOFF_P_R 10
#define TERSOFF_P_D_CUT 11
#define TERSOFF_P_LAMBDA1 12
#define TERSOFF_P_A 13

/* Maximum number of species per context. */
#define TERSOFF_MAX_SPECIES 4

/* Create a context computing in `precision` (TERSOFF_FP64 or TERSOFF_MIXED)
 * on the current CUDA device. *ctx receives the new context. */
int tersoff_create(tersoff_ctx** ctx, int precision);

/* Free a context and all device memory it owns. NULL is accepted. Waits for
 * the context's outstanding work. */
int tersoff_destroy(tersoff_ctx* ctx);

/* One-line description of the last failure on `ctx` (static storage owned by
 * the context; valid until the next call on it). */
const char* tersoff_last_error(const tersoff_ctx* ctx);

/* Switch the arithmetic path of an existing context. */
int tersoff_set_precision(tersoff_ctx* ctx, int precision);

/* Load the per-triplet parameter table (Eq. 5-7's parameters; Sec. III).
 * table: HOST array of n_species^3 records of TERSOFF_NPARAM doubles, record
 * ((ti*n_species + tj)*n_species + tk) for centre species ti, bond partner tj
 * and third atom tk. Record (ti,tj,tj) gives the pair terms of bond i-j
 * (n, beta, lambda2, B, lambda1, A and the R, D of f_C(r_ij)); record
 * (ti,tj,tk) gives the three-body terms (m, gamma, lambda3, c, d, h and the
 * R, D of f_C(r_ik)). m must be a positive integer; D > 0; n > 0.
 * The table is copied; the caller keeps ownership. */
int tersoff_params(tersoff_ctx* ctx, int n_species, const double* table);

/* Build the full ("skin") neighbour list S_i = { j != i : r_ij <= r_list }
 * (Sec. II Eq. 4, with the skin of Sec. III) for n atoms at positions x
 * (device, N x 3) with species types (device, N), in the periodic box `box`
 * (host, 3 doubles). r_list is the cutoff plus skin. The membership test is
 * exact: d = x_j - x_i; d -= L * rint(d * (1/L)) per axis in double, and
 * r^2 = (dx*dx + dy*dy) + dz*dz compared with r_list^2, all without fused
 * multiply-add. The list is kept inside the context and used by the compute
 * and MD calls until the next build. If an atom has more neighbours than the
 * current capacity, the capacity is grown and the build redone. Synchronises
 * `stream` (to read the overflow check). Returns TERSOFF_E_BOX_TOO_SMALL if
 * some box edge < 2 r_list and TERSOFF_E_NONFINITE for non-finite input.
 * Does not modify x. At most 2^26 atoms. */
int tersoff_neighbor_build(tersoff_ctx* ctx, const double* x, const int* types, int n,
                           const double* box, double r_list, void* stream);

/* Neighbour lists of a batch of n_systems independent periodic systems held
 * in one context (for fitting over many configurations; the paper treats one
 * system, Sec. II Eq. 4 applied to each). The atoms of system s are
 * x[offsets[s] .. offsets[s+1]) (device, N x 3 in total; types device, N);
 * sys_offsets: HOST, n_systems + 1 ints from 0 to n, non-decreasing; boxes:
 * HOST, n_systems x 3 orthorhombic edges, each at least 2 r_list
 * (TERSOFF_E_BOX_TOO_SMALL otherwise). Membership is the exact test of
 * tersoff_neighbor_build within each system; list entries hold global atom
 * indices (tersoff_neighbor_export works unchanged). Afterwards the context
 * is in batch mode: use tersoff_compute_batched and tersoff_backward (with one
 * gE per system); tersoff_compute and the MD calls return TERSOFF_E_STATE
 * until the next tersoff_neighbor_build. Synchronises `stream`. */
int tersoff_neighbor_build_batched(tersoff_ctx* ctx, const double* x, const int* types, int n,
                                   const int* sys_offsets, const double* boxes, int n_systems,
                                   double r_list, void* stream);

/* Energy, forces and virial of every system of the batch in one launch over
 * all atoms (Eq. 1, Eq. 5-7 per system). Outputs (device): energies[n_systems],
 * forces[N x 3], virials[n_systems x 6] (component order as tersoff_compute);
 * any may be NULL. Per-system sums are formed in a fixed order. */
int tersoff_compute_batched(tersoff_ctx* ctx, const double* x, int n, double* energies,
                            double* forces, double* virials, void* stream);

/* Current per-atom capacity of the neighbour list and the largest count seen
 * in the last build (host outputs, either may be NULL). */
int tersoff_neighbor_capacity(const tersoff_ctx* ctx, int* capacity, int* max_count);

/* Set the per-atom capacity used by the next build (>= 1). */
int tersoff_set_neighbor_capacity(tersoff_ctx* ctx, int capacity);

/* Copy the last-built list out: cnt (device, N int32) receives each atom's
 * neighbour count, nbr (device, N x cap int32, row-major) the neighbour indices
 * in ascending order, padded with -1. Returns TERSOFF_E_NEIGH_OVERFLOW if some
 * count exceeds cap (cnt is still written). */
int tersoff_neighbor_export(tersoff_ctx* ctx, int* cnt, int* nbr, int cap, void* stream);

/* Energy, forces and virial (Eq. 1, Eq. 5-7) of the atoms of the last
 * neighbour build, at positions x (device, N x 3; the same atoms, moved by
 * less than half the skin since the build). Outputs (device): energy[1],
 * forces[N x 3], virial[6] = (xx, yy, zz, xy, xz, yz) with
 * W_ab = sum over terms of (x_a - x_i)_a F_b relative to each term's centre
 * atom i (positive = repulsive); any output may be NULL. Outputs are
 * overwritten, not accumulated. */
int tersoff_compute(tersoff_ctx* ctx, const double* x, int n, double* energy,
                    double* forces, double* virial, void* stream);

/* Adjoint of tersoff_compute (for fitting the parameters). The paper has no
 * backward pass; this is the derivative of Eq. 5-7 with respect to the table
 * entries and the positions. For the weights gE (device, 1 double: the
 * derivative of the caller's loss with respect to E) and gF (device, N x 3,
 * the derivative with respect to the forces; NULL means zero):
 *   grad_table (device, n_species^3 x TERSOFF_NPARAM doubles, table layout)
 *       = d/dtheta [ gE E + sum_a gF_a . F_a ]      (field m gets 0: integer)
 *   grad_x (device, N x 3) = d/dx [ gE E + sum_a gF_a . F_a ]
 *       = -gE F - H gF,   H the Hessian d^2E/dx^2 (a Hessian-vector product;
 *       with gF == NULL only the -gE F term).
 * The three-body sums are recomputed, not stored by the forward call. Either
 * output may be NULL. x: positions of the atoms of the last neighbour build
 * (as for tersoff_compute). Arithmetic follows the context's precision (mixed:
 * per-term float, gradient sums in double). In batch mode (see
 * tersoff_neighbor_build_batched) gE holds one weight per system and E is the
 * vector of system energies: grad_table = d/dtheta [sum_s gE_s E_s +
 * sum_a gF_a . F_a] and grad_x = -gE_{s(a)} F_a - (H gF)_a. */
int tersoff_backward(tersoff_ctx* ctx, const double* x, int n, const double* gE,
                     const double* gF, double* grad_x, double* grad_table, void* stream);

/* Largest atom count accepted by tersoff_compute_noalloc. */
#define TERSOFF_NOALLOC_MAX_ATOMS 65536

/* The energy, forces and virial of tersoff_compute (same arguments, same
 * results up to rounding order), computed without allocating any memory in
 * this call. The paper has no counterpart: this is a library facility.
 *
 * Who needs it: callers that must not ask the CUDA runtime for memory while
 * they run. Examples are a program that has handed nearly all device memory
 * to its own pool (an allocation could fail, or force that pool to give memory
 * back), and a latency-sensitive loop sharing the GPU with other streams
 * (freeing device memory waits for the whole device). tersoff_compute may
 * allocate per-neighbour buffers on its first call and after a precision or
 * capacity change; this call allocates no device memory. (With kernel timing
 * on, tersoff_set_timing, it records event pairs in a host-side list, which
 * can allocate host memory.)
 *
 * How: forces are added with FP64 atomics (as with TERSOFF_SCATTER_ATOMIC,
 * whatever the context's scatter mode) into a scratch array of fixed size
 * that is part of the library (one per device, about 1.5 MiB), then copied to
 * the outputs. The context's scatter mode and the TERSOFF_ABLATE_FP32_SUMS
 * switch (which act on the gather of tersoff_compute) therefore do not apply;
 * the other ablation switches do. The first call on a device looks up that
 * array's address (and makes the CUDA runtime load the library's device code
 * there if it has not yet) and keeps it for the life of the process; make that
 * first call before any stream capture. A device reset (cudaDeviceReset) after
 * that first call is not supported: the kept address would be stale.
 *
 * Limits: n <= TERSOFF_NOALLOC_MAX_ATOMS, else TERSOFF_E_INVALID_ARG with
 * nothing enqueued. Every call on a device, from any context, uses the same
 * scratch array: two calls whose work overlaps on the GPU (different streams
 * without an ordering between them) race and give wrong results. Each call
 * clears the parts it accumulates into before use. The context must hold a
 * neighbour list built for these atoms (tersoff_neighbor_build, which does
 * allocate). */
int tersoff_compute_noalloc(tersoff_ctx* ctx, const double* x, int n, double* energy,
                            double* forces, double* virial, void* stream);

/* Per-atom energy of the last tersoff_compute (device, N doubles): the pair
 * terms V(i, j, zeta_ij) summed over j, assigned to the centre atom i. */
int tersoff_compute_peratom(tersoff_ctx* ctx, const double* x, int n, double* eatom,
                            void* stream);

/* rebuild_every value of the MD calls: rebuild the neighbour list when some
 * atom has moved more than half the skin (r_list minus the largest cutoff)
 * since the last build, the validity limit of the skin list (Sec. III). The
 * check runs on the device after every step; inside a CUDA graph the rebuild
 * is a conditional node, so no host synchronisation is needed. */
#define TERSOFF_REBUILD_ON_SKIN (-1)

/* Velocity-Verlet NVE steps in metal units (x in A, v in A/ps, dt in ps,
 * forces in eV/A). Requires a prior tersoff_neighbor_build on these atoms and
 * forces f holding F(x) (for example from tersoff_compute). Each step:
 *   v += dt/2 f/m;  x += dt v;  rebuild the list when the number of steps
 *   since the last build reaches rebuild_every (0 = never; or, with
 *   TERSOFF_REBUILD_ON_SKIN, when an atom has moved more than half the skin);
 *   f = F(x);  v += dt/2 f/m.
 * mass: HOST array of n_species masses (amu). x, v, f (device, N x 3) are
 * updated in place; positions are not wrapped into the box. thermo (device,
 * nsteps x 3, may be NULL) receives potential, kinetic and total energy (eV)
 * after each step. Synchronises `stream` at the end to report neighbour
 * overflow during the run. */
int tersoff_md_step(tersoff_ctx* ctx, double* x, double* v, double* f, int n,
                    const double* mass, double dt, int nsteps, int rebuild_every,
                    double* thermo, void* stream);

/* The same MD steps with HOST arrays x, v, f (N x 3 doubles each, ideally
 * pinned) and host thermo (nsteps x 3, may be NULL): copies the state to the
 * device, runs tersoff_md_step, and copies x, v, f and thermo back. Device
 * staging buffers are owned by the context. Synchronises `stream`. */
int tersoff_md_step_host(tersoff_ctx* ctx, double* x, double* v, double* f, int n,
                         const double* mass, double dt, int nsteps, int rebuild_every,
                         double* thermo, void* stream);

/* MD checkpoints (the paper has no counterpart: its runs use LAMMPS, whose
 * restart files it does not discuss; a facility of this library for long
 * runs such as the 10^6-step accuracy experiment of Sec. V-D).
 *
 * tersoff_checkpoint_save writes to the host file `path` (created or
 * truncated) one line of JSON text, then raw little-endian arrays in this
 * order: the species (int32, n), the parameter table (double,
 * n_species^3 x TERSOFF_NPARAM, as given to tersoff_params), x, v and f
 * (double, n x 3 each). The header holds the format name and version, n,
 * n_species, the precision, the box, the list radius, the caller's step
 * counter `step`, the number of MD steps since the last neighbour build (the
 * phase of tersoff_md_step's fixed rebuild period), the neighbour-list
 * capacity per atom and the context's launch
 * options (scatter mode, tersoff_set_launch's waves, split and block, lanes,
 * ablation flags, graphs), which decide the order of the sums. x, v, f: device,
 * N x 3 (f = F(x), as tersoff_md_step leaves it). Requires tersoff_params and
 * a single-system tersoff_neighbor_build on these n atoms (TERSOFF_E_STATE
 * otherwise); TERSOFF_E_INVALID_ARG when the file cannot be written.
 * Synchronises `stream`. */
int tersoff_checkpoint_save(tersoff_ctx* ctx, const char* path, const double* x, const double* v,
                            const double* f, int n, long long step, void* stream);

/* Atom and species counts of the checkpoint file `path` (host outputs, either
 * may be NULL); TERSOFF_E_INVALID_ARG when the file is missing or is not a
 * checkpoint of this format and version. Needs no context. */
int tersoff_checkpoint_info(const char* path, int* n, int* n_species);

/* Restores a checkpoint into ctx and the caller's device arrays x, v, f
 * (N x 3 double) and types (N int32): sets the saved precision, parameter
 * table, launch options and list capacity, copies the state, builds the neighbour list of the saved positions
 * with the saved box and list radius, and restores the phase of the rebuild
 * period, so that tersoff_md_step continues the saved run. When the
 * checkpoint was taken right after a list rebuild (zero steps since the
 * build, as after md_step calls whose step count is a multiple of
 * rebuild_every) the list is the one the uninterrupted run built at that
 * step, and with the gather scatter the continued trajectory equals the
 * uninterrupted one (the same sequence of calls) bit for bit; otherwise it
 * agrees to rounding. *step (host, may be NULL) receives the saved step
 * counter. n must equal the saved count; TERSOFF_E_INVALID_ARG for another
 * count, a missing, truncated or foreign file. Synchronises `stream`. */
int tersoff_checkpoint_load(tersoff_ctx* ctx, const char* path, double* x, double* v, double* f,
                            int* types, int n, long long* step, void* stream);

/* Autotuner (the paper has no counterpart; its launch choices are made for
 * CPUs). Times the context's launch options on its current system and keeps
 * the fastest:
 *   - the force scatter (tersoff_set_scatter);
 *   - the separate register-capacity-8 launch on a side stream
 *     (automatic / never / whenever needed);
 *   - the lanes per atom of the main force launch (tersoff_set_lanes);
 *   - the force kernel's grid: one thread per atom, or 1, 2 or 4 waves of
 *     the blocks resident on all multiprocessors looping over the atoms;
 *   - the block size of the pack, integrate and gather kernels (128/256/512).
 * One option at a time, the others fixed at their best so far (coordinate
 * descent); every trial is the median of 5 timed repetitions (CUDA events on
 * `stream`) after 2 untimed ones. The winner then replaces the context's
 * starting options only if a confirming pair of trials (9 repetitions each)
 * finds it at least 1% faster.
 * With v != NULL the repetition is one tersoff_md_step call of `steps` steps
 * (list rebuilt after the last step) on internal copies of x and v (device,
 * N x 3, not modified), mass (host) and dt as for tersoff_md_step; afterwards
 * the neighbour list is rebuilt at x. With v == NULL the repetition is one
 * force evaluation at x (tersoff_compute, or tersoff_compute_batched for a
 * batch). Requires a neighbour build; synchronises `stream`; allocates
 * scratch for the copies during the call. */
int tersoff_autotune(tersoff_ctx* ctx, const double* x, const double* v, int n,
                     const double* mass, double dt, int steps, void* stream);

/* Sets the launch options that tersoff_autotune chooses: waves (0 = one
 * thread per atom in the force kernel, else that many waves of resident
 * blocks, at most 64), split (-1 automatic, 0 never, 1 whenever bucket 1 is
 * non-empty) and block (pack / integrate / gather block size, a power of two
 * in [64, 512]). Results do not depend on them beyond rounding order. */
int tersoff_set_launch(tersoff_ctx* ctx, int waves, int split, int block);

/* Lanes per centre atom in the main force launch (mixed path, one or two
 * species, single systems; the FP64 path and batches always use one thread
 * per atom): 4 = one lane per bond, four lanes per atom, the neighbourhood
 * shared by warp shuffles (the paper's scheme (a) of Sec. IV-B, bonds on
 * vector lanes), atoms with more than four bonds inside the cutoffs finished
 * by a per-thread launch; 1 = one thread per atom with the bonds in registers
 * (scheme (c)); 0 (the default) = automatic, which is 1 (measured faster on the
 * Si benchmark). Results agree to rounding order; tersoff_autotune also tries
 * 4 and keeps it when it is faster. */
int tersoff_set_lanes(tersoff_ctx* ctx, int lanes);

/* Ablations of the paper's design choices, for measurement (results are
 * unchanged up to rounding order; the default is 0):
 *   TERSOFF_ABLATE_NO_SHORT   no stored short list: every force evaluation
 *                             filters the full skin list by the cutoffs (the
 *                             per-step filter of Sec. IV-D) and scatters forces
 *                             with FP64 atomics (slots need the short list);
 *   TERSOFF_ABLATE_GENERAL    every atom takes Algorithm 2's loops over its list
 *                             with the three-body terms recomputed in the second K
 *                             loop, instead of the register-resident neighbourhood
 *                             with pre-computed derivatives (Sec. IV-A);
 *   TERSOFF_ABLATE_FP32_SUMS  mixed path, gather scatter: each atom's force is
 *                             the plain float sum of its contributions (the
 *                             single-precision accumulation of the paper's
 *                             all-single mode, Sec. V-E) instead of the
 *                             compensated float pair carried into double. This
 *                             one changes results beyond rounding order: it
 *                             measures what the compensated sums buy;
 *   TERSOFF_ABLATE_FASTFWD    no list filtering at all: one lane per centre atom
 *                             walks the full skin list, each lane moving its own
 *                             J (and, inside, K) index forward to the next entry
 *                             inside the cutoff while the ready lanes wait, the
 *                             body running once a warp vote finds every lane
 *                             ready (the fast-forward scheme of Sec. IV-C, Fig. 2,
 *                             with the warp vote of the paper's CUDA back-end,
 *                             Sec. VI-B); forces through FP64 atomics. Single
 *                             systems only (batches ignore it). */
#define TERSOFF_ABLATE_NO_SHORT 1
#define TERSOFF_ABLATE_GENERAL 2
#define TERSOFF_ABLATE_FP32_SUMS 4
#define TERSOFF_ABLATE_FASTFWD 8
/* TERSOFF_ABLATE_COMP_ATOM_SUMS (mixed path, one species, single systems; a
 * variant rather than a removal): the sums that one thread forms over the
 * terms of its centre atom -- the force on each neighbour and on the atom,
 * the atom's energy and virial, at most z(z-1) + z terms each -- are carried
 * as compensated float pairs (TwoSum) and converted into double, and forces
 * are scattered with FP64 atomics (whatever the scatter mode): every sum is
 * then exact to double rounding beyond the float terms themselves, the strict
 * reading of the paper's mixed mode (Sec. V-E). By default those per-atom sums
 * are plain float; this switch measures what that costs. Atoms on the general
 * path (more bonds than the register capacity) keep float per-atom sums. */
#define TERSOFF_ABLATE_COMP_ATOM_SUMS 16
int tersoff_set_ablation(tersoff_ctx* ctx, int flags);

/* One-line text of the last tersoff_autotune: the chosen options and every
 * trial's time (storage owned by the context). */
const char* tersoff_autotune_summary(const tersoff_ctx* ctx);

/* Number of neighbour rebuilds during the last tersoff_md_step call on this
 * context (host output). */
int tersoff_md_rebuilds(const tersoff_ctx* ctx, int* count);

/* Force scatter. TERSOFF_SCATTER_GATHER (default): every atom stores the
 * force its own terms put on each short-list neighbour in a slot of that
 * neighbour (plain stores), and the force on an atom is gathered from its own
 * slots in a fixed order, summed with exact error compensation
 * (mixed path; the rounding error of every float addition is carried and
 * added in double) or in double (FP64 path): deterministic, no atomics.
 * TERSOFF_SCATTER_ATOMIC: every force contribution is added to the force
 * array with FP64 atomics. Results agree to rounding; speed differs by
 * workload (the benchmark measures both). */
#define TERSOFF_SCATTER_GATHER 0
#define TERSOFF_SCATTER_ATOMIC 1
int tersoff_set_scatter(tersoff_ctx* ctx, int mode);

/* MD execution mode. With enable != 0 (the default) tersoff_md_step records
 * its whole sequence of steps (integration, neighbour rebuilds, forces) once
 * as a CUDA graph and replays it on later calls with the same arguments and
 * context state; the state is snapshotted before each replay and, if a
 * rebuild inside it exceeded the list capacity, restored and the steps rerun
 * with host-checked rebuilds. With enable == 0 every step is launched
 * directly. */
int tersoff_set_graphs(tersoff_ctx* ctx, int enable);

/* Number of kernel launches this context has enqueued since creation (host
 * output); used to report launch counts. */
int tersoff_launch_count(const tersoff_ctx* ctx, long long* count);

/* Kernel timing. With enable != 0 the context records a CUDA event pair on the
 * launching stream around every force-kernel launch (kind 0), every neighbour
 * build (kind 1, all of its kernels) and every integration kernel (kind 2).
 * Enabling resets the totals. */
int tersoff_set_timing(tersoff_ctx* ctx, int enable);

/* Accumulated device time in milliseconds and number of timed launches of
 * `kind` since timing was enabled (host outputs). Waits for the recorded
 * events. */
int tersoff_timing(tersoff_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Arithmetic-pipe peaks of the current device, measured by loop kernels (the
 * paper reports run times only; these are the denominators of the force
 * kernels' rooflines). Runs five short kernels on `stream` (about 10 ms in
 * all), each the median of 5 event-timed launches after an untimed one:
 * chains of FP32 fused multiply-adds, of FP64 fused multiply-adds, and of the
 * special-function unit's rsqrt, ex2 and lg2. out: HOST array of 6 doubles
 * receiving FP32 TFLOP/s (an FMA counts 2), FP64 TFLOP/s, rsqrt, ex2 and lg2
 * rates in 1e12 operations/s, and the multiprocessor count. Allocates a
 * scratch buffer for the kernels' results during the call; synchronises
 * `stream`. Returns TERSOFF_E_CUDA when no device is usable. */
int tersoff_pipe_peaks(double* out, void* stream);

/* Ghost-shell packing for a slab decomposition of one periodic cell over
 * ranks (the data-parallel layout of the paper's multi-node runs, Sec. V):
 * one rank's owned atoms in; its local frame and the two face sets it sends
 * to its neighbours out, each already in the receiver's local frame, so that
 * a halo exchange sends the buffers as they are and the receiver appends
 * them after its own atoms.
 *   x (n x 3), types (n, int32), ids (n, int64): the rank's owned atoms.
 *   axis: the cut axis (0, 1 or 2).
 *   geo: HOST array of 9 doubles: L (the box edge along the axis), lo, hi
 *     (the rank's slab [lo, hi)), r_ghost (the ghost width), frame (the
 *     origin of the rank's local frame along the axis), shift_lower,
 *     frame_lower, shift_upper, frame_upper (for the lower / upper face set:
 *     the periodic shift it takes across the boundary, and the frame origin
 *     of the neighbour that receives it).
 * With u the axis coordinate wrapped into [0, L) (the remainder of the
 * division by L, moved up by L when negative; +0 for a zero remainder):
 *   x_local (n x 3): the owned atoms with the axis coordinate u - frame;
 *   set 0 (lower face: u - lo < r_ghost) and set 1 (upper face:
 *   hi - u <= r_ghost), each in ascending owned index, into send_x
 *   (2 x cap x 3, set-major), send_t (2 x cap) and send_id (2 x cap), the
 *   axis coordinate (u + shift) - frame of the receiver (two roundings, in
 *   that order), the other two coordinates unchanged;
 *   counts (2 ints): the sizes of the two sets (atoms beyond cap are counted,
 *   not written: compare counts with cap).
 * Needs no parameters or lists on ctx (it serves error reporting and the
 * launch count). Allocates a scratch buffer of 8 bytes per 1024 atoms
 * (stream-ordered); does not synchronise. */
int tersoff_halo_pack(tersoff_ctx* ctx, const double* x, const int* types, const long long* ids,
                      int n, int axis, const double* geo, int cap, double* x_local,
                      double* send_x, int* send_t, long long* send_id, int* counts,
                      void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TERSOFF_GB300_H */
