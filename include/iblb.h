/*
 * iblb.h -- C ABI of the GB300 (sm_103a) immersed-boundary lattice-Boltzmann library.
 *
 * One coupled IB-LB time step of arXiv:2305.18919, Sec. III, in the paper's order:
 *   1. nodal forces phi = phi^S + phi^V + phi^W on every mesh vertex   (Eqs. 2, 16-19)
 *   2. spreading F(x) = sum_i phi_i delta_D(x - q_i)                   (Eqs. 13-15)
 *   3. BGK collision with Guo forcing, then streaming with half-way
 *      bounce-back walls in z and periodic x, y                         (Eqs. 9-10)
 *   4. fluid velocity u = (sum_i c_i f_i + F/2) / rho                   (Sec. III, Guo shift)
 *   5. interpolation qdot_i = sum_x u(x) delta_D(x - q_i)               (Eq. 11)
 *   6. Euler update q_i += qdot_i                                       (Eq. 12)
 *
 * Conventions shared by every call:
 *  - Lattice units (dx = dt = 1). Layers z = 0 and z = nz-1 are solid wall nodes; the fluid is
 *    z = 1 .. nz-2 and the bounce-back planes are z = 0.5 and z = nz-1.5. With z_periodic = 1
 *    there are no walls and every layer is fluid.
 *  - Host arrays are row-major, x fastest: scalar fields [nz][ny][nx], vector fields
 *    [nz][ny][nx][3], populations [19][nz][ny][nx], vertices [nv][3], faces [nf][3].
 *  - Inputs are copied; the caller keeps ownership of every pointer it passes. Outputs are
 *    written to caller-owned buffers, always in double precision.
 *  - Every call returns 0 on success or a negative IBLB_E* code; iblb_last_error() then holds a
 *    one-line message. All device work is ordered on the stream given to iblb_create();
 *    calls that return data to the host synchronise that stream.
 *  - The library allocates its own device memory with cudaMalloc and frees it in
 *    iblb_destroy(). No call falls back to the CPU.
 *  - D3Q19 ordering inside the library is private; populations are exchanged in the order
 *    0 rest, 1..6 = +x,-x,+y,-y,+z,-z, 7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),
 *    (+1,0,+1),(-1,0,-1),(+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 */
#ifndef IBLB_H
#define IBLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBLB_OK 0
#define IBLB_EINVAL (-1)    /* bad argument: sizes, tau <= 1/2, open or inconsistent mesh */
#define IBLB_ENOMEM (-2)    /* device allocation failed */
#define IBLB_ECUDA (-3)     /* a CUDA runtime call failed (message names it) */
#define IBLB_EUNSTABLE (-4) /* health check failed: NaN, |qdot| >= 0.1, vertex within 0.05 of a
                               wall plane, or |V/V0 - 1| > 0.05 */
#define IBLB_ECAPACITY (-5) /* an internal bound was exceeded (active-tile table) */
#define IBLB_ETIMEOUT (-6)  /* a bounded wait inside a kernel gave up (the staged stream-collide
                               pass, iblb_set_stage_wait_limit); the context stays usable */

#define IBLB_FP64 1 /* populations and interface arithmetic in double */
#define IBLB_FP32 2 /* populations (stored as f_i - w_i rho0) and interface forces in float;
                       vertex positions and the volume sum stay in double */
#define IBLB_FP16 3 /* as IBLB_FP32, but populations stored in IEEE half precision as
                       (f_i - w_i rho0) * 1024 / w_i; collision and forcing in float */
#define IBLB_BF16 4 /* as IBLB_FP16 with bfloat16 storage of (f_i - w_i rho0) / w_i */

typedef struct iblb_ctx iblb_ctx;

/* Lattice description (Sec. III; walls: Sec. III last paragraph; moving walls: Sec. IV). */
typedef struct {
  int32_t nx, ny, nz;      /* nx, ny multiples of 4; nz >= 3 with walls, >= 4 periodic */
  int32_t precision;       /* IBLB_FP64, IBLB_FP32, IBLB_FP16 or IBLB_BF16 */
  int32_t z_periodic;      /* 0: bounce-back walls at both z ends; 1: periodic z (tests) */
  int32_t ib_sms;          /* SMs given to the interface chain of iblb_step as a partition of
                              the GPU (green context); the stream-collide passes get the rest.
                              0: when the stream-collide pass moves at least 1 GiB
                              (2 x 19 x nx ny nz x storage bytes) 24, 40 with 16-bit
                              storage and none with FP64; below that 64 (rounded to the device's
                              partition granularity), < 0: no
                              partition (both share all SMs, interface stream at top priority).
                              If the device or driver cannot partition, no partition is used. */
  double tau;              /* BGK relaxation time, > 1/2 (viscosity (tau - 1/2)/3) */
  double rho0;             /* reference density (initial state and moving-wall term) */
  double wall_u_bottom[3]; /* wall velocity at z = 0.5 (tangential components only) */
  double wall_u_top[3];    /* wall velocity at z = nz - 1.5 */
  double body_force[3];    /* uniform body force density added to the IB force */
} iblb_lattice_desc;

/* Interface parameters of one mesh: Eq. 2 (alpha), Eq. 18 (kV), Eq. 19 (eps, xi). */
typedef struct {
  double alpha[3];         /* (alpha1 pre-stress, alpha2 dilatation, alpha3 shear) */
  double kV;               /* volume-force coefficient (the paper fixes 1) */
  double eps;              /* Lennard-Jones strength */
  double xi;               /* Lennard-Jones length (the paper fixes 0.5) */
  int32_t wall_force_on;   /* apply Eq. 19 against both wall planes */
  int32_t volume_force_on; /* apply Eq. 18 */
} iblb_iface_params;

/* Create a lattice at rest, f = f^eq(rho0, 0) (Eq. 10). `cuda_stream` is a cudaStream_t (NULL:
   the legacy default stream). On success *out owns all device memory of the context. */
int iblb_create(const iblb_lattice_desc *desc, void *cuda_stream, iblb_ctx **out);

/* Release every resource of the context (NULL is accepted). Synchronises its stream. */
void iblb_destroy(iblb_ctx *ctx);

/* Message of the last failed call on this context ("" if none). Owned by the context. */
const char *iblb_last_error(const iblb_ctx *ctx);

/* Add the triangulated interface (Sec. III: refined icosahedron). verts [nv][3], faces [nf][3]
   oriented counter-clockwise seen from outside. The mesh must be closed and consistently
   oriented (every edge shared by exactly two faces in opposite directions, nf == 2 nv - 4);
   this shape becomes the reference shape (per-face metric, V0 = its volume). One mesh per
   context; *mesh_id receives 0. IBLB_EINVAL otherwise. */
int iblb_add_mesh(iblb_ctx *ctx, const double *verts, int32_t nv, const int32_t *faces,
                  int32_t nf, int32_t *mesh_id);

/* Set alpha, kV, eps, xi and the force switches of a mesh (defaults: all alpha 0, kV 1,
   eps 0, xi 0.5, wall force off, volume force on). */
int iblb_set_interface(iblb_ctx *ctx, int32_t mesh_id, const iblb_iface_params *params);

/* Replace the current vertex positions (host [nv][3]); the reference shape is unchanged. */
int iblb_set_vertices(iblb_ctx *ctx, int32_t mesh_id, const double *q);

/* Set every fluid node to f^eq(rho, u) (Eq. 10) of host fields rho [nz][ny][nx] and
   u [nz][ny][nx][3]; values on wall layers are ignored. */
int iblb_init_equilibrium(iblb_ctx *ctx, const double *rho, const double *u);

/* Advance nsteps coupled steps (order above). Work is queued on the stream; the call
   synchronises to read the health word every `every` steps of iblb_set_health_interval (1000
   by default) and at its end, and returns IBLB_EUNSTABLE or IBLB_ECAPACITY if a check failed
   during the steps read so far (the steps done then stop at the end of that interval),
   IBLB_ETIMEOUT if a bounded wait of the staged stream-collide pass gave up. */
int iblb_step(iblb_ctx *ctx, int32_t nsteps);

/* Steps between health-word reads in iblb_step: every >= 1, or 0 for one read at the end of
   each call. IBLB_EINVAL for every < 0. */
int iblb_set_health_interval(iblb_ctx *ctx, int32_t every);

/* Advance nsteps coupled steps like iblb_step, queued on the stream without any
   synchronisation: the health word is not read by this call. A failed check of these steps is
   returned (IBLB_EUNSTABLE, IBLB_ECAPACITY, IBLB_ETIMEOUT) by the next call that reads it:
   iblb_read_vertices, iblb_read_vertex_velocities, iblb_read_fields, iblb_read_forces or
   iblb_read_volume (in the same synchronisation as their own transfer; their output is
   written all the same), iblb_check_health, iblb_step, iblb_read_force_field, the adjoint
   calls or iblb_batch_step (before doing their own work, or in its status). Repeated calls
   keep the first failure until it is read. iblb_init_equilibrium and iblb_load_state discard
   an unread failure with the state. For a loop that exchanges data with the host every step
   (set vertices, step, read vertices) this leaves one synchronisation per step.
   IBLB_EINVAL for nsteps < 0. */
int iblb_step_async(iblb_ctx *ctx, int32_t nsteps);

/* Read the health word of steps queued by iblb_step_async (synchronises); IBLB_OK if there
   are none or they passed, else the failure as iblb_step reports it. */
int iblb_check_health(iblb_ctx *ctx);

/* rho [nz][ny][nx] and u [nz][ny][nx][3] of the current post-streaming state; u carries half
   of the force of the last spreading step (none before the first step) plus the body force.
   Wall-layer nodes report rho0 and their wall velocity. */
int iblb_read_fields(iblb_ctx *ctx, double *rho, double *u);

/* Same as iblb_read_fields into device buffers rho_dev [nz][ny][nx] and u_dev [nz][ny][nx][3]
   (doubles, caller-owned, e.g. torch tensors), ordered on the context's stream; does not
   synchronise. */
int iblb_read_fields_device(iblb_ctx *ctx, double *rho_dev, double *u_dev);

/* Populations [19][nz][ny][nx] of the current post-streaming state (wall layers: 0). */
int iblb_read_populations(iblb_ctx *ctx, double *f);

/* Vertex positions [nv][3] (Eq. 12) of the current state. */
int iblb_read_vertices(iblb_ctx *ctx, int32_t mesh_id, double *q);

/* Same as iblb_read_vertices into a device buffer `q_dev` ([nv][3] doubles, caller-owned),
   ordered on the context's stream; does not synchronise. */
int iblb_read_vertices_device(iblb_ctx *ctx, int32_t mesh_id, double *q_dev);

/* Vertex velocities [nv][3] interpolated in the last step (Eq. 11); zero before any step. */
int iblb_read_vertex_velocities(iblb_ctx *ctx, int32_t mesh_id, double *qdot);

/* Nodal forces phi [nv][3] (Eq. 16) evaluated now at the current vertex positions. */
int iblb_read_forces(iblb_ctx *ctx, int32_t mesh_id, double *phi);

/* Force density F [nz][ny][nx][3] (Eq. 13) spread now from the forces at the current vertex
   positions (the interface part only; the body force is not included). */
int iblb_read_force_field(iblb_ctx *ctx, double *F);

/* Current enclosed volume V (Eq. 18, sum over faces, accumulated in double) and V0. */
int iblb_read_volume(iblb_ctx *ctx, int32_t mesh_id, double *V, double *V0);

/* Write / read the full state (populations, vertices, reference shape, parameters, step
   count) to / from a binary file. load_state requires a context created with the same
   lattice description and a mesh of the same size. */
int iblb_save_state(iblb_ctx *ctx, const char *path);
int iblb_load_state(iblb_ctx *ctx, const char *path);

/* Number of steps taken so far. */
int64_t iblb_steps_done(const iblb_ctx *ctx);

/* Profiling of the dominant kernel. When on, iblb_step() brackets every stream-collide launch
   with CUDA events on the context's stream. iblb_profile() synchronises and returns the summed
   stream-collide time in milliseconds, the number of stream-collide launches and the number of
   kernel launches made by iblb_step() since profiling was switched on. */
int iblb_set_profiling(iblb_ctx *ctx, int32_t on);
int iblb_profile(iblb_ctx *ctx, double *k1_ms, int64_t *k1_launches, int64_t *kernel_launches);

/* Enclosed volume of a closed, outward-oriented triangle mesh, for callers that cannot allocate
   device memory. The paper has no counterpart: this is a library service. It computes
   V = sum over faces of (x0 - c) . ((x1 - x0) x (x2 - x0)) / 6 in double, the same volume the
   interface forces use (iblb_read_volume), from caller-owned device arrays: q_dev [nv][3]
   doubles, faces_dev [nf][3] int32 (indices into q_dev), centre = host pointer to 3 doubles
   (any fixed point; a point near the mesh limits rounding), V_dev = device pointer to one
   double that receives V. Work is queued on `cuda_stream` (a cudaStream_t, NULL = legacy
   default stream); the call does not synchronise.
   Nothing is allocated: the only scratch is a 32 KB array of per-block partial sums that the
   library holds on every device that loads it, until the process exits. Callers in a host
   framework that owns all device memory, or in a loop that must not pay for cudaMalloc's
   device-wide synchronisation, can use it. Every call looks up that array's device address in
   the caller's current context (so the call stays correct under a non-primary context and
   after cudaDeviceReset); the first call on a device also loads the library's device code into
   that context, so make the first call before any stream capture begins.
   Limits and errors: nf <= 1,048,576 (IBLB_ECAPACITY beyond), nf >= 1 and non-NULL pointers
   (IBLB_EINVAL otherwise), IBLB_ECUDA if a launch fails. Every call shares the one array and
   overwrites the partials it uses, so calls that overlap on the GPU (on different streams)
   race and must be ordered by the caller. */
int iblb_mesh_volume_noalloc(const double *q_dev, const int32_t *faces_dev, int32_t nf,
                             const double *centre, double *V_dev, void *cuda_stream);

/* ---- Batched ensemble ----------------------------------------------------------------------
   Many independent contexts (lattices and meshes of any sizes) advanced together. The paper
   runs one box at a time; this is the ensemble form of its parameter sweeps (Sec. V), a library
   service with no counterpart in the paper.

   iblb_batch_create makes n contexts, instance i from descs[i], each with its own CUDA stream,
   and returns the batch in *out. With descs[0].ib_sms > 0 the batch splits the GPU's SMs as a
   single context does, that many SMs for the interface kernels of every instance and the rest
   for the stream-collide passes; 0 or < 0 (the default, the faster on ensembles of many
   meshes) or a device that cannot partition gives no partition. The other descriptors' ib_sms
   are ignored. The contexts are configured and read through the
   single-context calls on the handles that iblb_batch_context returns (borrowed: they stay
   owned by the batch and are released by iblb_batch_destroy, which synchronises).
   `cuda_stream` (a cudaStream_t, NULL: legacy default stream) orders the batch against the
   caller's work.

   iblb_batch_step advances every instance by nsteps coupled steps (the iblb_step sequence).
   Each kernel of a step is one launch over all instances of a precision (up to 256 per
   launch), whose blocks read their instance's arguments from tables the batch builds at its
   first use and again after any instance was reconfigured (mesh, interface parameters,
   initial state, kernel choice) or stepped alone by an odd count; steps run in pairs, and a
   freshly initialised instance takes its first step, and an odd last step is taken, through
   the single-context kernels. The call synchronises once at its end and reads every
   instance's health word: it returns the first failing instance's IBLB_EUNSTABLE /
   IBLB_ECAPACITY (message in iblb_batch_last_error) and iblb_batch_status fills status[n]
   with each instance's result. Results are identical, bit for bit, to stepping each context
   alone.

   iblb_batch_tune picks, per distinct lattice shape and precision, the lattice rows per block
   (1, 2 or 4, within 128 threads) of the single-context stream-collide pass (the first and odd
   steps) by timing `trials` launches of each on the instance's own stream (the state is not
   advanced); iblb_batch_k1_rows reports the choice. */
typedef struct iblb_batch iblb_batch;
int iblb_batch_create(const iblb_lattice_desc *descs, int32_t n, void *cuda_stream,
                      iblb_batch **out);
void iblb_batch_destroy(iblb_batch *batch);
const char *iblb_batch_last_error(const iblb_batch *batch);
int32_t iblb_batch_size(const iblb_batch *batch);
iblb_ctx *iblb_batch_context(iblb_batch *batch, int32_t i); /* NULL if i is out of range */
int iblb_batch_tune(iblb_batch *batch, int32_t trials);
int32_t iblb_batch_k1_rows(const iblb_batch *batch, int32_t i);
int iblb_batch_step(iblb_batch *batch, int32_t nsteps);
int iblb_batch_status(const iblb_batch *batch, int32_t *status);

/* ---- Adjoint: gradients of an observable of the final vertex positions ----------------------
   The discrete adjoint of the coupled step (Sec. III) with respect to the interface parameters
   theta = (alpha1, alpha2, alpha3, eps) of Eq. 2 and Eq. 19; IBLB_FP64 or IBLB_FP32 contexts
   with a mesh. The forward run is the context's own; the reverse pass is in double, and with
   FP32 storage it linearises the double-precision step about the recomputed FP32 trajectory
   (the copies keep the populations as stored, so the recomputation repeats it bit for bit).

   iblb_adjoint_record advances nsteps steps from the current state (as iblb_step would) and keeps
   a copy of the state (populations and positions) every `every` steps on the device: memory
   ceil(nsteps/every) + 1 copies of the state. The context is left at the end of the run.

   iblb_adjoint_gradient takes dJdq (host [nv][3]: the derivative of an observable J with respect
   to the final positions) and writes dJdtheta (host [4]). It runs the recorded steps backwards:
   each segment is recomputed forward from its copy (every + 1 more states on the device), then
   the transposed step is applied state by state. The context is returned to the end of the run;
   the recording stays valid for further calls with other dJdq.

   iblb_adjoint_release frees the recording and the work arrays (iblb_destroy also does).
   Errors: IBLB_EINVAL (16-bit storage, no mesh, nothing recorded, nsteps or every < 1), the health
   errors of iblb_step during the record or the recomputation, IBLB_ENOMEM, IBLB_ECUDA. */
int iblb_adjoint_record(iblb_ctx *ctx, int32_t nsteps, int32_t every);
int iblb_adjoint_gradient(iblb_ctx *ctx, const double *dJdq, double *dJdtheta);
int iblb_adjoint_release(iblb_ctx *ctx);

/* Kernel of the full-lattice stream-collide pass (pull streaming with Eqs. 9-10) from the
   second step of a run on (the first step after an initialisation reads the state in place and
   always takes the direct kernel).
   IBLB_STREAM_COLLIDE_STAGED: a persistent kernel, one block per SM of the lattice partition.
     The lattice is cut into units of `rows` consecutive lattice rows (y) of one layer (z); one
     warp of each block copies what the next units pull, 19 blocks of `rows` population rows,
     into shared memory with bulk asynchronous copies completing on mbarriers, `stages` buffers
     deep, and `warps` compute warps collide from there. Applies to IBLB_FP32, IBLB_FP16 and
     IBLB_BF16 when nx values of the storage type are a whole number of 16-byte blocks and two
     buffers fit in shared memory; otherwise the direct kernel runs.
   IBLB_STREAM_COLLIDE_DIRECT: every thread loads its nodes' populations from global memory.
   IBLB_STREAM_COLLIDE_AUTO (default): staged for 16-bit storage, direct otherwise (the faster
     of the two on GB300 for each storage type).
   Both kernels give the same populations bit for bit. stages: 0 (4) or 2..8, reduced to what
   fits in shared memory; warps: 0 (8) or 1..16 (at most 8 with four nodes per lane); rows: 0
   (as many as keep one copy within 4 KB) or a power of two up to 16 that divides ny; nodes:
   nodes per compute lane with 16-bit storage, 0 (the default), 2 or 4 (FP32 always takes 2).
   IBLB_EINVAL for anything else. A staged block whose wait for its copies gives up (after
   1 s) returns early, and iblb_step then returns IBLB_ETIMEOUT. */
#define IBLB_STREAM_COLLIDE_AUTO 0
#define IBLB_STREAM_COLLIDE_STAGED 1
#define IBLB_STREAM_COLLIDE_DIRECT 2
int iblb_set_stream_collide(iblb_ctx *ctx, int32_t kind, int32_t stages, int32_t warps,
                            int32_t rows, int32_t nodes);
/* Limit in nanoseconds of each wait of the staged kernel's warps for a buffer to fill or to be
   released, on the GPU's global timer (default 1e9, range 0 .. 6e10; 0: a single non-blocking
   test, so that a block's first wait, which comes before its copies complete, gives up; this
   exercises the timeout path). A wait that runs out records the timeout in the health word
   and its block stops; before the block exits, its copying warp still waits up to 1 s for the
   copies it has in flight. iblb_step then returns IBLB_ETIMEOUT and the populations of that
   step are incomplete; the context stays usable (iblb_init_equilibrium or iblb_load_state restore
   a state). IBLB_EINVAL outside the range. */
int iblb_set_stage_wait_limit(iblb_ctx *ctx, int64_t ns);

/* 1 if the stream-collide steps after the first take the staged kernel (as configured by
   iblb_set_stream_collide for this lattice and storage type), 0 for the direct kernel, -1 for
   a NULL context. */
int32_t iblb_stream_collide_staged(const iblb_ctx *ctx);

/* SMs of the interface partition of iblb_step (0: no partition, -1: NULL context). */
int32_t iblb_interface_sms(const iblb_ctx *ctx);

/* Bytes moved per fluid cell by one stream-collide launch (19 loads + 19 stores of the
   population storage type): 304 for IBLB_FP64, 152 for IBLB_FP32, 76 for IBLB_FP16 and
   IBLB_BF16. */
int64_t iblb_bytes_per_cell(const iblb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* IBLB_H */
