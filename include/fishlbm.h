/*
 * fishlbm.h -- C ABI of the B300 (sm_103a) library that advances FishGym's
 * fluid solver (arXiv 2206.01683, Sec. III-B "GPU-accelerated localized
 * fluid-structure interaction"): one lattice Boltzmann time step on a D3Q27
 * lattice, carried in the robot's accelerating local frame (the fictitious
 * force of Eq. 3), closed by non-equilibrium extrapolation on the open faces
 * of the moving domain (Sec. III-B "Simulation"), and two-way coupled to the
 * uniformly sampled robot surface (Sec. III-B "Simulation", the external
 * force tau_ext of Eq. 1) by a direct-forcing immersed boundary.
 *
 * Units are lattice units (dx = dt = 1, c_s^2 = 1/3).  Cell centres sit at
 * integer coordinates 0..n-1 per axis; cell index c = x + nx*(y + ny*z).
 *
 * Conventions shared by every call:
 *  - Every call returns an fg_status; fg_last_error() gives a thread-local
 *    message for the last failure.  No C++ exception crosses the ABI.
 *  - The library owns all device memory of a domain.  Caller buffers (host or
 *    device) are only read or written during the call, except where a call
 *    says it is asynchronous.
 *  - All GPU work of a domain runs on the CUDA stream given at creation
 *    (NULL = the legacy default stream).  fg_step is asynchronous; calls that
 *    return data to the host synchronise that stream first.
 *  - On an error the domain is unchanged, except FG_ERR_NUMERIC, which marks
 *    the domain poisoned until fg_init_fields resets its state.
 */
#ifndef FISHLBM_H
#define FISHLBM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fg_domain fg_domain; /* opaque, owned by the library */

typedef enum {
    FG_OK = 0,
    FG_ERR_INVALID = -1,  /* bad argument; nothing was changed */
    FG_ERR_CUDA = -2,     /* a CUDA runtime call failed (message in fg_last_error) */
    FG_ERR_OOM = -3,      /* device allocation failed */
    FG_ERR_TIMEOUT = -4,  /* a bounded device wait gave up */
    FG_ERR_NUMERIC = -5,  /* NaN/Inf in the mass or force reduction; domain poisoned */
    FG_ERR_STATE = -6     /* call not valid in the domain's current state */
} fg_status;

/* Storage type of the populations.  Arithmetic is FP32 in every case; FP16
 * and BF16 store f_i - w_i (the deviation from the rest state) scaled by a
 * fixed power of two per velocity class. */
typedef enum { FG_F32 = 0, FG_F16 = 1, FG_BF16 = 2 } fg_storage;

/* Face condition.  Periodic faces come in pairs.  The three open kinds are
 * closed by non-equilibrium extrapolation from the inward neighbour (Sec.
 * III-B "Simulation"): a velocity inlet imposes u_in, an outflow imposes the
 * density rho0 and extrapolates u, a free-slip wall extrapolates u with its
 * normal component removed.  Boundary nodes are the outermost cell layer of
 * a non-periodic face; where faces meet, x-faces govern. */
typedef enum { FG_PERIODIC = 0, FG_VELOCITY = 1, FG_OUTFLOW = 2, FG_FREESLIP = 3 } fg_bc;

typedef struct {
    int nx, ny, nz;   /* cells per axis; >= 3 along a non-periodic axis */
    double tau;       /* BGK relaxation time, > 0.5; nu = (tau - 1/2)/3 */
    int face[6];      /* fg_bc for faces -x, +x, -y, +y, -z, +z */
    double u_in[3];   /* inlet velocity of FG_VELOCITY faces */
    double rho0;      /* initial density, and the density FG_OUTFLOW imposes */
    double u0[3];     /* initial velocity */
} fg_env_desc;

/* Stream-collide kernel: AUTO picks STAGED when every row has at most 512
 * cells, else PLAIN (and with the autotune option, the fastest candidate).
 * STAGED stages the source rows of each row group in shared memory with bulk
 * copies (persistent, double-buffered), 256 slots per population when rows
 * fit, else 512; STAGED512 forces 512.  PLAIN reads global memory directly,
 * one thread per cell (two where every row length is even).  FUSED runs the
 * whole step but its final reduction in one persistent launch: the IB
 * phases (stamping the marker stencils, node moments, interpolation and
 * spreading) and PLAIN's cell update taken from one work queue, so that cell
 * blocks no marker reaches (and, in a batch, other environments' blocks)
 * proceed while the IB phases run.  OVERLAP runs PLAIN with the IB beside it:
 * a small kernel stamps the markers' stencils and flags the PLAIN blocks they
 * fall in, a second, high-priority stream runs the IB kernel and then the
 * flagged blocks, while the domain's stream runs the other blocks.  All
 * compute the same step. */
typedef enum {
    FG_KERNEL_AUTO = 0,
    FG_KERNEL_PLAIN = 1,
    FG_KERNEL_STAGED = 2,
    FG_KERNEL_STAGED512 = 3,
    FG_KERNEL_FUSED = 4,
    FG_KERNEL_OVERLAP = 5
} fg_kernel_variant;

/* Population layout.  PULL keeps two population arrays: each step pulls
 * from one and writes the other.  AA keeps one array and updates it in place
 * (the AA access pattern: even steps read and write each cell's own slots,
 * odd steps read from and write to the neighbours' slots, with the
 * directions reversed between the two), halving population memory; it runs
 * the plain kernel (kernel_variant AUTO or PLAIN) and computes bit-identical
 * populations, forces and torques.  fg_step_state and the adjoint take PULL
 * only; the state buffers of fg_save_state, fg_load_state and fg_copy_state
 * have the same format in both layouts. */
typedef enum { FG_LAYOUT_PULL = 0, FG_LAYOUT_AA = 1 } fg_layout;

#define FG_MAX_IB_ITERS 8

typedef struct {
    int storage;        /* fg_storage */
    int layout;         /* fg_layout */
    int deterministic;  /* 1: the IB spread sums each node's contributions as
                           64-bit fixed-point integers (multiples of 2^-48,
                           exact and order-independent), so every step is
                           bit-reproducible; 0: FP32 vector atomics (the sum's
                           rounding depends on arrival order) */
    int ib_iters;       /* direct-forcing passes per step, 1..FG_MAX_IB_ITERS
                           (multi-direct forcing; each pass interpolates the
                           velocity corrected by the force spread in the
                           earlier passes, u~ + f_ib / (2 rho), and adds
                           2 R (U - U~) to the marker force).  The adjoint
                           takes 1 only. */
    int record_history; /* steps of (force, torque, mass) history kept on the
                           device per environment (0 = none), ring buffer */
    int kernel_variant; /* fg_kernel_variant */
    int autotune;       /* 1 (with kernel_variant AUTO): run fg_autotune at the
                           first fg_step (or fg_step_io / fg_step_state) with
                           n_steps > 0, so that it times the step with its
                           markers; that first call synchronises and must not
                           be made under stream capture */
    int ib_slip;        /* 1: slip (Neumann) direct forcing: only the normal
                           component of the marker slip is enforced,
                           dF = 2 R ((U - U~).n) n, with the unit normals given
                           by fg_set_marker_normals; 0: no-slip (default).  The
                           adjoint takes 0 only. */
    int eq_order;       /* 2: second-order (Hermite-2) equilibrium (default);
                           3: also the third-order terms D3Q27 carries,
                           4.5 w_i rho (c.u)((c.u)^2 - |u|^2), in the initial
                           state, the post-collision rebuild and the open-face
                           rule (removes the 3 u^2 error of the viscous
                           stress for shear along the flow).  The adjoint takes
                           2 only. */
    int use_graphs;     /* 1: each step is replayed from a captured CUDA graph
                           (captured on first use and whenever the marker count or
                           marker storage changes); 0: direct launches.  Steps taken
                           while fg_profile is on always launch directly.  Default
                           (opt == NULL): 1 */
} fg_options;

/* Frame motion of Eq. 3 for one environment: acc = translational
 * acceleration p'' of the frame, omega = its angular velocity (Eq. 3's r'),
 * domega = the rate of omega (r''), origin = the point x' is measured from.
 * The fictitious acceleration is -acc - domega x x' - omega x (omega x x')
 * - 2 omega x u. */
typedef struct {
    double acc[3], omega[3], domega[3], origin[3];
} fg_frame;

/* Create n_envs independent environments (n_envs > 1 is the batched form:
 * every environment advances in the same kernel launches).  opt may be NULL
 * (FP32, one pass, automatic kernel choice, graphs on).  cuda_stream is a cudaStream_t or NULL.  Populations are
 * initialised at equilibrium with (rho0, u0); the frame is at rest with its
 * origin at the domain centre.  Limits: 1 <= n_envs <= 4096; 1 <= cells
 * per axis <= 65536; P ny nz < 2^31 slots per environment (P = nx rounded up
 * to a multiple of 8).  Errors: FG_ERR_INVALID (sizes, limits, tau, rho0,
 * faces, options; checked before any GPU work), FG_ERR_OOM, FG_ERR_CUDA.
 * *out is set only on FG_OK. */
fg_status fg_create_domain(const fg_env_desc* envs, int n_envs, const fg_options* opt,
                           void* cuda_stream, fg_domain** out);

/* Copy the marker set of environment env: the robot surface sampled
 * uniformly before the simulation (Sec. III-B "Simulation").
 *   X[n][3]  positions (float, row-major), U[n][3] velocities at the current
 *   step, dV[n] surface weight of each marker (area x 1 lu), seg[n] segment
 *   id in [0, n_seg) (NULL: all 0), 1 <= n_seg <= 16, ref[3] the point
 *   torques are taken about (NULL: origin).
 * device_ptrs = 0: host arrays; 1: device arrays (copied on the stream,
 * asynchronously).  Host arrays in pinned (page-locked) memory are read in
 * place by a copy kernel on the stream, pageable ones are copied at the
 * call; either way the library keeps its own copy, and pinned or device
 * arrays must stay unchanged until the stream has reached the copy (as for
 * any asynchronous copy).  dV and seg may be NULL on later calls with the same n to
 * keep the previous values.  Periodic axes wrap X; along a non-periodic
 * axis every marker must satisfy 2 <= X < n-3 so its 4-point stencil stays
 * off the boundary layer: host arrays are checked here (FG_ERR_INVALID),
 * device arrays in the step kernel, which skips such a marker and reports
 * FG_ERR_INVALID from the next fg_get_body_force_torque. */
fg_status fg_set_markers(fg_domain* d, int env, int n, const float* X, const float* U,
                         const float* dV, const int* seg, int n_seg, const double ref[3],
                         int device_ptrs);

/* Index-check flags of a debug build (libfishlbm_debug.so, compiled with
 * -DFG_DEBUG_BOUNDS): bit set = some kernel computed an index outside its
 * array and skipped the access (1 pulled population, 2 emitted slot, 4 staged
 * bulk copy, 8 staged-row read, 16 IB stencil node, 32 reduction chunk,
 * 64 region cell).  reset != 0 clears them after reading.  Synchronises the
 * device.  A release build reports FG_ERR_STATE.  The paper has no
 * counterpart. */
fg_status fg_debug_flags(unsigned int* flags, int reset);

/* Failure-detection self test of the library's bounded device waits (the
 * mbarrier waits of the staged stream-collide kernel, the grid barrier of the
 * IB kernel, and the dependency wait of the fused step kernel's work queue),
 * run on conditions that never come: an mbarrier nobody arrives on, a grid
 * barrier whose target is never reached, a completion counter that stays
 * short.  Each wait gives up after `limit` polls (the step kernels use 2^22)
 * and reports instead of hanging or trapping: result[0] = 1 if the mbarrier
 * wait gave up, result[1] = 1 if the grid barrier gave up, result[2] = 1 if
 * the timeout bit was set in the status word, result[3] = 1 if the queue wait
 * gave up and set the queue's abort word (which stops the other blocks of a
 * fused launch).  result holds 4 ints.  Runs on the current device, allocates
 * and frees its own 60 bytes, synchronises; the context stays usable.  The
 * paper has no counterpart. */
fg_status fg_selftest_waits(unsigned int limit, int* result);

/* New positions and velocities for the markers of all environments at once
 * (the per-step update of a batch): X, U float [n][3], environment after
 * environment in the counts of each environment's last fg_set_markers, n their
 * total; host or device (device_ptrs).  Weights, segments and reference
 * points are unchanged.  One scatter launch (plus two copies for host
 * arrays) instead of one call per environment; asynchronous. */
fg_status fg_set_markers_all(fg_domain* d, int n, const float* X, const float* U, int device_ptrs);

/* Momentum and angular momentum of the fluid inside a sphere (centre,
 * radius; lattice units) in env's current state: out[0..2] = sum alpha j,
 * out[3..5] = sum alpha (x - centre) x j, with j = sum_i c_i f_i,
 * alpha = clamp(radius + 1/2 - |x - centre|, 0, 1) the cell's volume
 * fraction and x - centre the minimal image on periodic axes; *alpha_sum
 * (nullable) = sum alpha.  A free body's Newton-Euler equations need this
 * inner-fluid momentum every step (Eq. 1's tau_ext with the fluid inside the
 * immersed shell, Kempe & Froehlich 2012).  Compensated FP32 sums on the
 * device, added in FP64 on the host; synchronises. */
fg_status fg_region_momentum(fg_domain* d, int env, const double center[3], double radius, double* out,
                             double* alpha_sum);

/* Torque reference points of env's segment rows, refs[n_seg][3] (host),
 * n_seg equal to that of the last fg_set_markers: segment s reports its
 * torque about refs[s], so several bodies can share one marker set (each
 * body's segments about its own point, e.g. two fish of a school).  The
 * total row keeps the reference point of fg_set_markers.  refs = NULL returns
 * to that common point; fg_set_markers with a different n_seg does too.  The
 * call synchronises the stream. */
fg_status fg_set_segment_refs(fg_domain* d, int env, int n_seg, const double* refs);

/* A free rigid sphere advanced on the device: the body update of Eq. 1
 * (Sec. III-A) for a body whose only generalised forces are the fluid's
 * tau_ext, gravity and buoyancy, two-way coupled every step with no host
 * round trip.  Each step of the environment (fg_step, fg_step_io) then
 * places the n markers on the shell, X = c + R d_l, U = V + W x (X - c),
 * with torques about c; after the reduction it sums the momentum P and
 * angular momentum L of the fluid inside the shell (as fg_region_momentum)
 * and advances the body in FP64, with the inner fluid's change of momentum
 * (Kempe & Froehlich, J. Comput. Phys. 231, 2012):
 *   m_p dV = F + dP_in + (m_p - m_f) g,  I_p dW = T + dL_in,
 *   c += (V_old + V_new) / 2,
 * m_f = 4 pi R^3 / 3, m_p = density_ratio m_f, I_p = 0.4 m_p R^2, F and T
 * the environment's total force/torque row.  The body starts at rest at
 * center.  dirs[n][3] are unit directions (FP64, host), dV[n] the marker
 * weights (host); box_reaction = 1 adds -(m_p - m_f) g / (cells) to the
 * environment's frame acceleration (Eq. 3's acc term), so that in a closed
 * box the fluid carries the body's excess weight.  While attached, the
 * environment's markers, segment points and torque point follow the body:
 * fg_set_markers and fg_set_segment_refs on it, and fg_set_markers_all and
 * fg_step_io with marker arrays on the domain, fail with FG_ERR_STATE;
 * fg_init_fields leaves the body state alone.  One sphere per environment.
 * Errors: FG_ERR_INVALID (arguments, markers outside the domain's limits),
 * FG_ERR_STATE (a sphere attached already), FG_ERR_OOM, FG_ERR_CUDA.
 * Synchronises. */
fg_status fg_attach_sphere(fg_domain* d, int env, double radius, const double center[3], double density_ratio,
                           const double gravity[3], int n, const double* dirs, const float* dV, int box_reaction);
/* out[9] = centre, velocity, spin of the sphere attached to env (after the
 * steps enqueued so far; synchronises).  FG_ERR_STATE if none. */
fg_status fg_sphere_state(fg_domain* d, int env, double* out);
/* Detach the sphere of env (its markers stay where the last step put them;
 * the box reaction is removed from the frame).  FG_ERR_STATE if none. */
fg_status fg_detach_sphere(fg_domain* d, int env);

/* Unit surface normals of env's current markers for slip forcing
 * (fg_options.ib_slip = 1): N[n][3] float, host or device (device_ptrs), n
 * equal to the count given to the last fg_set_markers (normalised by the
 * caller; not rescaled).  They are copied and kept until replaced; a step of
 * a slip domain whose markers have no normals fails with FG_ERR_STATE, and
 * fg_set_markers with a new marker count drops them.  The paper applies a
 * slipping condition on immersed solids (Sec. III-B). */
fg_status fg_set_marker_normals(fg_domain* d, int env, int n, const float* N, int device_ptrs);

/* Advance every environment by n_steps time steps (asynchronous on the
 * domain's stream).  frames: NULL keeps the previous frames, else n_envs
 * fg_frame entries applied to all n_steps.  One step: interpolate the
 * post-stream velocity at the markers and spread the direct-forcing force;
 * stream, collide (regularized BGK + Guo forcing with the frame force) and
 * apply the open-face rule; reduce force, torque and mass (compensated FP32
 * pair sums on the device, evaluated in FP64 when read). */
fg_status fg_step(fg_domain* d, int n_steps, const fg_frame* frames);

/* Force and torque the fluid exerts on the body in environment env during the
 * last step (the tau_ext of Eq. 1), FP64: out[(n_seg + 1) * 6], one row
 * (Fx, Fy, Fz, Tx, Ty, Tz) per segment, then the total.  Synchronises the
 * stream.  Returns FG_ERR_NUMERIC if the step produced NaN/Inf. */
fg_status fg_get_body_force_torque(fg_domain* d, int env, double* out);

/* New markers and one step in one call, asynchronous: the positions and
 * velocities of all environments' markers (X and U float [n][3] as in
 * fg_set_markers_all: n the total of the counts of each environment's last
 * fg_set_markers, environment after environment; NULL keeps the current
 * ones), then fg_step(d, 1, frames).  Results equal those of
 * fg_set_markers_all followed by fg_step, bit for bit.  Where the step's IB
 * kernel is the cooperative k_ib_step (every kernel_variant but FUSED and
 * OVERLAP), no sphere is attached, and X, U are device arrays (device_ptrs =
 * 1) or pinned host arrays with at most two markers per warp of that kernel,
 * the arrays are not copied before the step: the IB kernel reads them in
 * its first phase and fills the domain's marker arrays from them (Sec. III-B:
 * the markers enter the step only through the interpolation stencils), which
 * saves the copy launch between steps.  Otherwise the call copies them first
 * as fg_set_markers_all does.  Either way the caller keeps X and U unchanged
 * until the step has run on the stream (as for any asynchronous copy).  The
 * same checks and errors as those calls; nothing is launched when a check
 * fails.  With the autotune option pending, it runs first (and synchronises). */
fg_status fg_step_markers(fg_domain* d, const float* X, const float* U, int device_ptrs, const fg_frame* frames);

/* One two-way coupled step in one call, for a loop in which the body's next
 * pose depends on the force just computed (Eq. 1): the new positions and
 * velocities of all environments' markers (as fg_set_markers_all: X and U
 * float [n][3], n the total of the counts of each environment's last
 * fg_set_markers, environment after environment; NULL keeps the current
 * ones), one step with `frames` (as fg_step with
 * n_steps = 1), then the force/torque rows of every environment read back
 * (as fg_get_body_force_torque, environment after environment: (n_seg_e + 1)
 * x 6 FP64 values each, so out holds sum_e (n_seg_e + 1) * 6).  X, U: host
 * or device (device_ptrs); frames, out: host.  The same checks and errors as
 * those calls; nothing is launched when a check fails.  The markers enter
 * the step as in fg_step_markers.  One synchronisation at the end (the step's
 * reduction writes the rows to mapped pinned memory, so no copy is issued). */
fg_status fg_step_io(fg_domain* d, const float* X, const float* U, int device_ptrs, const fg_frame* frames,
                     double* out);

/* Release all device memory of the domain; NULL is ignored. */
void fg_destroy(fg_domain* d);

/* Largest single device allocation the library may make, in bytes (0, the
 * default: no limit), process-wide.  A larger request fails with FG_ERR_OOM
 * as an exhausted device would, and the call that made it leaves its domain
 * unchanged (a failed fg_create_domain frees what it had allocated).  For
 * testing the out-of-memory paths without filling the device. */
fg_status fg_set_alloc_cap(unsigned long long bytes);

/* Thread-local message describing the last failed call ("" if none). */
const char* fg_last_error(void);

/* ---- state access (tests, checkpointing, diagnostics) ------------------ */

/* The library's velocity order: c[27][3] in {-1,0,1}, w[27]. */
fg_status fg_lattice(int* c, double* w);

/* Reset env's populations to equilibrium from host FP64 fields rho[ncell] and
 * u[ncell][3] (either NULL: rho0 / u0), clear the poisoned state.  Syncs. */
fg_status fg_init_fields(fg_domain* d, int env, const double* rho, const double* u);

/* Moments of env's stored post-collision state into host FP64 arrays:
 * rho[ncell] = sum_i f_i, u[ncell][3] = sum_i c_i f_i / rho (either NULL).
 * Synchronises. */
fg_status fg_get_fields(fg_domain* d, int env, double* rho, double* u);

/* Populations of env as host FP64 f[ncell][27] (library velocity order),
 * decoded from the storage type.  Synchronises. */
fg_status fg_get_populations(fg_domain* d, int env, double* f);

/* Overwrite env's populations from host FP64 f[ncell][27] (library velocity
 * order), rounded to the storage type.  Synchronises. */
fg_status fg_set_populations(fg_domain* d, int env, const double* f);

/* Marker force density F_l of the last step, host float F[n][3] (the fluid
 * receives F_l dV_l spread by the delta kernel).  Synchronises. */
fg_status fg_get_marker_force(fg_domain* d, int env, float* F);

/* Total mass sum_x rho after the last step: ncell + sum (rho - 1), the sum a
 * compensated FP32 pair on the device, evaluated in FP64.  Synchronises. */
fg_status fg_get_mass(fg_domain* d, int env, double* mass);

/* Mass-drift watchdog of env.  rel_tol > 0 takes env's current mass M0 as
 * the reference and makes the reduction of every later step check
 * |M - M0| <= rel_tol M0; a step that exceeds it sets status bit 3, and the
 * next call that reads results returns FG_ERR_NUMERIC ("mass drift") and
 * poisons the domain as a NaN does.  rel_tol <= 0 switches it off (the
 * default).  Periodic domains conserve mass to rounding; open faces exchange
 * mass, so there the tolerance bounds the net flux.  fg_init_fields keeps the
 * reference.  Synchronises. */
fg_status fg_watch_mass(fg_domain* d, int env, double rel_tol);

/* Copy up to max_steps rows of env's recorded history, oldest first; each row
 * is (n_seg + 1) * 6 force/torque values followed by the mass.  *n_rows gets
 * the number of rows written.  Synchronises. */
fg_status fg_get_history(fg_domain* d, int env, double* out, int max_steps, int* n_rows);

/* Raw device-format state of env for checkpoint/restore (the populations in
 * storage format, rows padded to a multiple of 8 cells): fg_state_bytes gives
 * the size; save copies it to a host buffer, load copies it back (both sync). */
fg_status fg_state_bytes(fg_domain* d, int env, unsigned long long* bytes);
fg_status fg_save_state(fg_domain* d, int env, void* host_buf);
fg_status fg_load_state(fg_domain* d, int env, const void* host_buf);

/* Device-to-device copy of env's raw state (fg_state_bytes bytes, the
 * populations in storage format) to (to_buf = 1) or from (to_buf = 0) a
 * caller device buffer, asynchronous on the stream (checkpoints). */
fg_status fg_copy_state(fg_domain* d, int env, void* buf, int to_buf);

/* One step of a single-environment domain from the caller's device state
 * buffer `in` into `out` (each fg_state_bytes bytes in the layout of
 * fg_copy_state; distinct): the step fg_step takes with the domain's markers,
 * frame (frames: NULL keeps the last) and options, force/torque, mass and
 * history recorded as by fg_step, but the domain's own populations are
 * neither read nor written.  Asynchronous on the stream.  Checkpoint
 * recompute steps from buffer to buffer with it, so no state is copied. */
fg_status fg_step_state(fg_domain* d, const void* in, void* out, const fg_frame* frames);

/* Device status word (bit 0 numeric, bit 1 invalid marker, bit 2 timeout,
 * bit 3 mass drift)
 * without clearing it.  Synchronises. */
fg_status fg_get_status(fg_domain* d, int* status);

/* Number of time steps taken since creation or the last fg_init_fields. */
fg_status fg_step_count(fg_domain* d, long long* steps);

/* ---- discrete adjoint ---------------------------------------------------
 * For gradients of losses built from the body force/torque rows with respect
 * to the marker positions and velocities (hence, through the caller's
 * skinning, the swimmer's joint-wave parameters).  Single environment, FP32
 * storage, periodic faces; frame forces included.  The domain keeps the
 * adjoint state lam = dL/df* (all zero after fg_adjoint_reset, the terminal
 * condition of a loss that does not read the final state).  The caller
 * replays the steps backwards: before the adjoint of step n it puts the
 * state f*^n into the domain (fg_copy_state / checkpoint + recompute), or
 * passes it in a buffer (fg_step_state / fg_adjoint_step_state), and sets
 * the step's markers (fg_set_markers); then fg_adjoint_step turns lam^{n+1}
 * into lam^n and writes the step's marker gradients.  The forward state is
 * not changed. */
fg_status fg_adjoint_reset(fg_domain* d);

/* frames: the step's frame (NULL keeps the last one); gF: host, (n_seg + 1) * 6
 * loss gradient w.r.t. the step's force/torque rows as fg_get_body_force_torque
 * reports them (NULL: none); gX, gU: device float [n][3] outputs, dL/dX_l and
 * dL/dU_l of this step.  Asynchronous on the stream. */
fg_status fg_adjoint_step(fg_domain* d, const fg_frame* frames, const double* gF, float* gX, float* gU);

/* fg_adjoint_step with the step's forward state f*^n read from the caller's
 * device buffer `state` (fg_state_bytes, the layout of fg_copy_state) instead
 * of the domain's populations. */
fg_status fg_adjoint_step_state(fg_domain* d, const void* state, const fg_frame* frames, const double* gF,
                                float* gX, float* gU);

/* The adjoint state lam as host FP64 [ncell][27] (library velocity order):
 * read it, or overwrite it (tests).  Both synchronise. */
fg_status fg_get_adjoint(fg_domain* d, double* lam);
fg_status fg_set_adjoint(fg_domain* d, const double* lam);

/* ---- timing ------------------------------------------------------------- */

/* Kernel ids for the timing calls. */
enum { FG_K_IB = 0, FG_K_STREAM_COLLIDE = 1, FG_K_REDUCE = 2, FG_K_COUNT = 3 };

/* enable != 0: record a CUDA event pair around every kernel launch of
 * fg_step (on the domain's stream); 0: stop.  Clears the accumulated times. */
fg_status fg_profile(fg_domain* d, int enable);

/* Sum of the recorded kernel durations (ms) and launch counts per kernel id
 * since fg_profile(d, 1) or the previous read; clears them.  Synchronises. */
fg_status fg_profile_read(fg_domain* d, double* ms, long long* launches);

/* Stream-collide variants (the autotuner's candidates). */
enum {
    FG_K1_PLAIN = 0,
    FG_K1_STAGED256 = 1,
    FG_K1_STAGED512 = 2,
    FG_K1_FUSED = 3,
    FG_K1_OVERLAP = 4,
    FG_K1_NVARIANTS = 5
};

/* Time every stream-collide variant that can run this domain's rows with the
 * step's IB work (the IB kernel and the variant's kernel; the fused kernel
 * does both), three interleaved rounds of five passes each, on the domain's
 * own buffers with its current markers: the populations, the step count and
 * the marker forces are not changed.  Keep the fastest, where a staged
 * variant must be more than 2% faster (whole steps favour the plain kernel by
 * about that much where the two are level in this timing).  choice
 * (nullable) gets the FG_K1_* kept; ms (nullable, FG_K1_NVARIANTS entries)
 * the mean pass time of each in its fastest round, -1 where not runnable.
 * Synchronises; graphs are recaptured on the next step. */
fg_status fg_autotune(fg_domain* d, int* choice, double* ms);

/* The FG_K1_* variant in use. */
fg_status fg_stream_collide_variant(fg_domain* d, int* variant);

/* Algorithmic bytes one launch of the stream-collide kernel moves: 27 reads
 * and 27 writes of a population per cell of every environment. */
fg_status fg_stream_collide_bytes(fg_domain* d, unsigned long long* bytes);

/* ---- allocation-free body force -----------------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need the body force: a program
 * whose device memory is wholly owned by another framework's pool, or a
 * control loop that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree imply.
 *
 * fg_body_force_noalloc computes, for a step that starts from the state g,
 * the post-stream velocity interpolated at the markers (Peskin 4-point
 * delta, frame half-force shift), the direct-forcing marker force F_l =
 * 2 R_l (U_l - U~_l), and the force and torque on the body, FP64.  That is
 * what fg_step reports through fg_get_body_force_torque for a domain with
 * one no-slip direct-forcing pass (ib_iters = 1, ib_slip = 0) whose segment
 * rows are all taken about ref (no fg_set_segment_refs); it is not that for
 * other domains.  It does not spread the force or advance the fluid.  It
 * allocates nothing: its scratch (one float triple per marker and a flag
 * word) is a static device array of FG_NOALLOC_MAX_MARKERS markers, about
 * 0.8 MB, that every GPU loading this library holds until the process exits.
 *   env     grid size and faces (tau, u_in, rho0, u0 are not used)
 *   g       device, FP32, the populations in the library's storage layout:
 *           f_i - w_i as g[27][nz][ny][P], P = nx rounded up to a multiple of
 *           8, velocity order of fg_lattice (what fg_save_state returns for
 *           an FP32 domain)
 *   X, U    device, float [n][3]; dV device float [n]; seg device int [n] in
 *           [0, n_seg) or NULL; 1 <= n_seg <= 16; ref[3] host (NULL: origin),
 *           the point every row's torque is taken about
 *   frame   host, or NULL for a frame at rest with origin at the centre
 *   out     device, double [(n_seg + 1) * 6]: one row per segment, then the
 *           total; NaN rows if a marker lay outside its allowed range
 *           (2 <= X < n-3 along non-periodic axes)
 * Runs asynchronously on cuda_stream (a cudaStream_t, NULL = legacy default).
 * The first call on a device looks up the scratch's device address with that
 * device current; make that first call before any stream capture.  Later
 * calls outside a capture look it up again (a context created anew, after a
 * device reset, is then served at its own address); a call under capture
 * uses the address found last, and fails with FG_ERR_STATE if there is none.
 * Every call uses the same scratch, which keeps the last call's contents
 * (each call clears the flag word before use): calls that overlap on the GPU
 * (on different streams, or from different threads) race and must be
 * serialised by the caller.  n > FG_NOALLOC_MAX_MARKERS is rejected with
 * FG_ERR_INVALID. */
#define FG_NOALLOC_MAX_MARKERS 65536
fg_status fg_body_force_noalloc(const fg_env_desc* env, const float* g, const float* X, const float* U,
                                const float* dV, const int* seg, int n, int n_seg, const double ref[3],
                                const fg_frame* frame, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FISHLBM_H */
