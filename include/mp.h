/*
 * mp.h -- C ABI of libmp, the GB300 (sm_103a) library for the sorption-modified
 * moment-propagation (MP) method of Levesque, Duvail, Pagonabarraga, Frenkel and
 * Rotenberg, "Accounting for adsorption and desorption in Lattice Boltzmann simulations"
 * (arXiv:1303.2470), and for the BGK lattice-Boltzmann solve that provides its flow.
 *
 * Conventions shared by every entry point
 *  - Lattice units: dx = dt = 1. D3Q19 velocities (19 discrete velocities, Sec. "Algorithm").
 *  - Lattice layout: node n = x + nx*(y + ny*z), x fastest; every axis is periodic.
 *    Solid walls or grains are solid nodes of the mask.
 *  - Velocity fields are FP32, structure of arrays: u[0..N) = u_x, u[N..2N) = u_y,
 *    u[2N..3N) = u_z, zero on solid nodes.
 *  - Pointers documented as "device" must be CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory. Nothing is retained after a call
 *    returns unless stated.
 *  - Every function returns MP_OK (0) or a negative status, and never aborts the process.
 *    The thread-local text of the last failure is returned by mp_last_error().
 *  - Work is enqueued on the stream given in the options (NULL = the legacy default
 *    stream). Calls that return results to host memory synchronise that stream.
 */
#ifndef MP_H
#define MP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define MP_OK 0
#define MP_EINVAL (-1)        /* an argument is out of range or inconsistent             */
#define MP_ENOMEM (-2)        /* a device or host allocation failed                       */
#define MP_ECUDA (-3)         /* a CUDA runtime call or kernel launch failed              */
#define MP_ENEGPROB (-4)      /* a link probability or a stay fraction is negative        */
#define MP_ENOTCONVERGED (-5) /* lb_steady: max_steps reached above tol, or unstable      */
#define MP_ETIMEOUT (-6)      /* a bounded device-side wait gave up                       */

/* ---- memory location of a caller pointer --------------------------------------------- */
#define MP_HOST 0
#define MP_DEVICE 1

/* ---- storage / arithmetic precision of the propagated fields ------------------------- */
#define MP_FP32 0 /* FP32 storage and arithmetic, FP64 reductions and D(t) (default)        */
#define MP_FP64 1 /* FP64 storage, arithmetic and reductions                                */
/* IEEE binary16 storage of the fields with FP32 arithmetic and FP64 reductions (no
 * counterpart in the paper: a storage variant that halves the bytes of every field access).
 * Stored values are scaled per species by the partition function Z_s = N_F + K N_I, so the
 * equilibrium free density is stored as 1 (no subnormal densities), and narrowed to binary16
 * after every update either stochastically (MP_ROUND_STOCHASTIC: rounded up in magnitude
 * with probability equal to the dropped fraction of the spacing, with random bits from a
 * counter-based hash of the step and the element, so the rounding is unbiased and
 * reproducible) or to nearest (MP_ROUND_NEAREST, which loses every per-step change below
 * half a spacing). Z, D, mp_mass and the field I/O are unscaled. Needs K = k_a/k_d <= 30000
 * (adsorbed values must stay below the binary16 maximum); not available in groups. */
#define MP_FP16 2

/* ---- rounding of binary16 storage (mp_options.rounding) ------------------------------- */
#define MP_ROUND_STOCHASTIC 0
#define MP_ROUND_NEAREST 1

/* ---- initial density field ------------------------------------------------------------ */
#define MP_INIT_EQUILIBRIUM 0 /* Boltzmann weights of Sec. "Algorithm" (free + adsorbed)    */
#define MP_INIT_UNIFORM 1     /* 1/N_fluid on every free fluid node, nothing adsorbed       */

#define MP_MAX_SPECIES 32 /* species (D_b, k_a, k_d sets) sharing one medium and flow      */

/* ---- evaluation of the step (mp_options.scheme) --------------------------------------- */
/* X + the sum of exactly antisymmetric net link fluxes, every product correctly rounded, so
 * that both ends of a link see opposite fluxes: total mass changes only by the final rounding
 * of each node's update (and not at all for a stationary field). FP64, FP32 and FP16. */
#define MP_SCHEME_FLUX 0
/* The paper's direct form X' = sum_i p_i(r - c_i) X(r - c_i) + (1 - sum_i p_i(r) - p_a) X(r)
 * + p_d X_a (Eq. propagated_quantity with Eqs. Pads, newP), with the incoming link
 * probabilities (one species) or their flow-dependent parts (several species), the
 * outgoing sums and u*_g of every fluid node tabulated once by mp_init (about 80 bytes per
 * fluid node). FP32 only. Link probabilities are bitwise those of MP_SCHEME_FLUX; total mass
 * is conserved up to the FP32 rounding of each node's outgoing sum (a relative error below
 * 2^-25 of X(r) per step, of random sign across the nodes of a porous medium; in media with
 * few distinct nodes, such as slits, it adds up coherently). With several species the fields
 * are stored for the fluid nodes only (in the order of the sorted fluid list; mp_get_field
 * and mp_set_field still exchange dense arrays), which takes the porosity's share of the
 * memory of the flux scheme's dense fields. */
#define MP_SCHEME_DIRECT 1

/* A medium: the solid mask of an nx*ny*nz periodic lattice. */
typedef struct {
    int nx, ny, nz;       /* >= 3 each, nx*ny*nz <= 2^31 - 256                               */
    const uint8_t* solid; /* nx*ny*nz bytes, nonzero = solid node                            */
    int location;         /* MP_HOST or MP_DEVICE: where `solid` lives                       */
} mp_geometry;

/* Options of an MP context; mp_default_options() fills the defaults. */
typedef struct {
    int precision;      /* MP_FP32 (default), MP_FP64 or MP_FP16                             */
    int directions;     /* velocity moments to propagate, bit mask 1 = x, 2 = y, 4 = z;
                           0 means x only                                                   */
    int init_density;   /* MP_INIT_EQUILIBRIUM (default) or MP_INIT_UNIFORM                 */
    int allow_negative; /* 0: negative link probabilities fail mp_init with MP_ENEGPROB;
                           1: they are only counted (see mp_info). A negative stay fraction
                           always fails.                                                    */
    int64_t capacity;   /* time points kept in the device Z(t)/D(t) series, >= 2;
                           0 means 131072. mp_step fails once the series is full.           */
    void* stream;       /* cudaStream_t of all work of the context; NULL = default stream   */
    int rounding;       /* MP_FP16 only: MP_ROUND_STOCHASTIC (default) or MP_ROUND_NEAREST  */
    int scheme;         /* MP_SCHEME_FLUX (default) or MP_SCHEME_DIRECT                      */
    int autotune;       /* MP_SCHEME_DIRECT only. 0: run the variant given below. Nonzero:
                           mp_init times every variant (link table or link terms recomputed
                           from the flow; one launch per step or one persistent launch per run
                           of steps; blocks of 128, 256 or 512; several species also tiled)
                           for 20 steps on the initial
                           state, restores the state and keeps the fastest (needs 24 free
                           entries in the series). See mp_variant.                          */
    int variant;        /* MP_SCHEME_DIRECT without autotune: 0 (one launch per step, link
                           table, blocks of 256) or MP_VARIANT_* flags                       */
} mp_options;

/* ---- kernel variants of MP_SCHEME_DIRECT (mp_options.variant); all give the same fields ---- */
#define MP_VARIANT_RECOMPUTE 1  /* link terms recomputed from the packed flow, no link table   */
#define MP_VARIANT_PERSISTENT 2 /* one persistent launch per run of steps                       */
#define MP_VARIANT_BLOCK128 4   /* blocks of 128 threads (default 256)                          */
#define MP_VARIANT_BLOCK512 8   /* blocks of 512 threads                                        */
#define MP_VARIANT_TILED 16     /* several species: tiles of 32 x 8 lattice columns marched along
                                   z through shared memory (blocks of 128, link terms recomputed);
                                   ignored by contexts of one species                          */

void mp_default_options(mp_options* opt);

typedef struct mp_ctx mp_ctx;

/*
 * mp_init -- set up the MP of one tracer species in a medium with a steady flow.
 *
 * Paper: Sec. "Algorithm": link probabilities p_i = f_i/rho - w_i + w_i lambda Q / 2 with
 * Q = 1 and f_i/rho read as the D3Q19 equilibrium of the local velocity u; lambda = 12 D_b
 * (D_b = lambda c_s^2 dt / 4); p_a = k_a dt/dx, p_d = k_d dt; Boltzmann weights (free
 * 1/Z on the fluid, adsorbed K/Z on interfacial nodes, K = k_a/(k_d dx)); the velocity
 * moment after the first step. Links into solid nodes carry no probability. Interfacial
 * nodes are the fluid nodes with at least one solid D3Q19 neighbour.
 *
 *  out      receives the new context (host pointer to a handle); unchanged on failure.
 *  g        the medium; g->solid is copied, so it may be freed after the call.
 *  u        device, FP32, 3*N, SoA; NULL = fluid at rest. Copied at the call.
 *  D_b      bulk diffusion coefficient, 0 < D_b <= 1/8.
 *  k_a,k_d  adsorption (length/time) and desorption (1/time) rates, in [0, 1]; the
 *           equilibrium start needs k_d > 0 whenever k_a > 0.
 *  opt      options, NULL = defaults.
 * After the call the density and velocity-moment fields are at t = 1 and the series hold
 * Z(0), Z(1), D(0) = Z(0)/2, D(1) = D(0) + Z(1). Allocates all device memory of the context.
 * Errors: MP_EINVAL, MP_ENOMEM, MP_ECUDA, MP_ENEGPROB.
 */
int mp_init(mp_ctx** out, const mp_geometry* g, const float* u, double D_b, double k_a,
            double k_d, const mp_options* opt);

/*
 * mp_init_batch -- as mp_init for n_species species (1..MP_MAX_SPECIES) that share the
 * medium and the flow; D_b, k_a, k_d are host arrays of n_species values. All species
 * advance together in every mp_step.
 */
int mp_init_batch(mp_ctx** out, const mp_geometry* g, const float* u, int n_species,
                  const double* D_b, const double* k_a, const double* k_d,
                  const mp_options* opt);

/*
 * mp_step -- advance every species and field n >= 0 steps t -> t+1.
 *
 * Paper: Sec. "Algorithm", Eq. (propagated_quantity) for P*, Eq. (Pads) and Eq. (newP) for
 * the exchange with the adsorbed population on interfacial nodes, with the adsorbed share
 * removed from the stay fraction (1 - sum_i p_i - p_a) so that total mass is conserved;
 * then Z_g(t+1) = sum_r P_g(r,t+1) sum_i p_i(r) c_ig (last equation of that section) and
 * D(t+1) = D(t) + Z(t+1) (Eq. D_t_from_vacf as a sum over steps), both in FP64.
 * Asynchronous on the context's stream. On a context created with its own stream (not the
 * legacy or per-thread default stream), calls with n >= 128 replay runs of 64 steps from a
 * CUDA graph captured at first use (one per starting buffer): the same kernels with the
 * same arguments, so results are identical; it only removes the per-launch host cost.
 * With MP_SCHEME_DIRECT the variant chosen at mp_init runs (see mp_variant); a persistent
 * variant runs up to 2^20 steps per launch.
 * Errors: MP_EINVAL (n < 0, or the series would exceed its capacity), MP_ECUDA.
 */
int mp_step(mp_ctx* c, int64_t n);

/*
 * mp_vacf -- copy the series Z_g(t) and D_g(t), t = 0..T, of one species and direction to
 * host memory (synchronises the stream).
 *  species    0..n_species-1;  direction 0 = x, 1 = y, 2 = z (must be propagated).
 *  Z, D       host arrays of cap doubles each (either may be NULL).
 *  n_out      receives T+1, the number of time points available (may exceed cap; then
 *             only the first cap are written).
 * Errors: MP_EINVAL, MP_ECUDA.
 */
int mp_vacf(mp_ctx* c, int species, int direction, double* Z, double* D, int64_t cap,
            int64_t* n_out);

/*
 * mp_mass -- FP64 sums of the density field of one species (synchronises the stream):
 *  out[0] = sum over fluid nodes of P, out[1] = sum over interfacial nodes of Gamma
 *  (P_ads), out[2] = sum over interfacial nodes of P. Total mass out[0] + out[1] is
 *  conserved by the step; out[1]/out[2] tends to K = k_a/k_d at equilibrium.
 */
int mp_mass(mp_ctx* c, int species, double out[3]);

typedef struct {
    int64_t n_nodes;          /* N = nx*ny*nz                                           */
    int64_t n_fluid;          /* fluid nodes                                            */
    int64_t n_interface;      /* interfacial fluid nodes                                */
    int64_t n_negative_links; /* open links with p_i < 0, summed over species           */
    int64_t t;                /* current time of the fields (1 after mp_init)           */
    int n_species;
    int n_fields;             /* 1 + number of velocity moments                         */
    int precision;
} mp_info_t;

int mp_info(mp_ctx* c, mp_info_t* info);

/*
 * mp_get_field / mp_set_field -- copy one propagated field of one species between the
 * device and dense host arrays (for checks and checkpoints; synchronises the stream).
 *  field 0 = density P; field k >= 1 = k-th propagated velocity moment (x, y, z order).
 *  free_dense  host, N doubles: the free field (zero on solid nodes).
 *  ads_dense   host, N doubles or NULL: the adsorbed partner, zero off the interface.
 * mp_set_field ignores solid nodes and non-interfacial entries of ads_dense.
 */
int mp_get_field(mp_ctx* c, int species, int field, double* free_dense, double* ads_dense);
int mp_set_field(mp_ctx* c, int species, int field, const double* free_dense,
                 const double* ads_dense);

/*
 * Groups -- several contexts (media of any sizes, each with its own species) advanced
 * together, one kernel launch per step for all of them.
 *
 * Paper: the same step as mp_step (Sec. "Algorithm"); the paper treats one species in one
 * medium at a time, and a group only batches independent problems.
 *
 * mp_group_create
 *  out          receives the group handle.
 *  ctxs, n      1..16 distinct FP32 contexts with the same field layout (the same number of
 *               velocity moments, padded: 1 or 2-3). They keep their own streams, series
 *               and fields; while grouped, mp_step on them fails (use mp_group_step), and
 *               the group must be freed before any of them.
 *  graph_steps  even number of steps captured once into a CUDA graph and replayed for long
 *               runs (0 = plain launches). The group runs on its own internal stream,
 *               ordered after and before the contexts' streams with events.
 *  autotune     nonzero: time 20 steps at block sizes 128, 256 and 512 on a copy of the
 *               current state (restored afterwards) and keep the fastest; otherwise 256.
 *               Needs at least one free entry in every context's series.
 * mp_group_step advances every context n steps (same results as separate mp_step calls:
 * identical fields; Z and D equal up to the order of the FP64 block sums when the block
 * size differs from 256). mp_group_block_size returns the block size in use.
 * Contexts created with MP_SCHEME_DIRECT form a direct group (all of them must be): one
 * launch per step or one persistent launch per run of steps for all of them, the variant
 * autotuned as for mp_options.autotune when `autotune` is nonzero (graph_steps is then
 * unused: runs of 128 steps or more replay graphs of 64); mp_group_variant names it. With a
 * tiled variant (several species), Z and D equal separate mp_step calls up to the grouping
 * of its FP32 warp sums (about 1e-7 relative); the fields are identical.
 * mp_group_create_ex: the same with `variant` (MP_VARIANT_* flags) for a direct group
 * without autotune (flux groups ignore it); mp_group_create is mp_group_create_ex with 0.
 * Errors: MP_EINVAL, MP_ENOMEM, MP_ECUDA.
 */
typedef struct mp_group mp_group;
int mp_group_create(mp_group** out, mp_ctx* const* ctxs, int n, int graph_steps, int autotune);
int mp_group_create_ex(mp_group** out, mp_ctx* const* ctxs, int n, int graph_steps, int autotune, int variant);
int mp_group_step(mp_group* g, int64_t n);
int mp_group_block_size(mp_group* g);
const char* mp_group_variant(mp_group* g);
void mp_group_free(mp_group* g);

/*
 * mp_classify -- node classes of a medium, as used by every other entry point.
 *
 * Paper: Sec. "Algorithm", the three node classes of the Boltzmann weights: solid S, fluid F
 * and interfacial I (fluid nodes with at least one solid D3Q19 neighbour). Also marks the
 * largest cluster of fluid nodes connected by D3Q19 links (periodic), on which lb_steady
 * applies its body force (ties go to the cluster holding the smallest node index).
 *  g            the medium (host or device mask).
 *  cls          host, N bytes out: 0 solid, 1 fluid, 2 interfacial, plus 4 when the node is
 *               in the largest cluster.
 *  n_fluid, n_interface, n_cluster   host outputs (each may be NULL).
 *  stream       cudaStream_t or NULL; synchronised before return.
 * Errors: MP_EINVAL, MP_ENOMEM, MP_ECUDA.
 */
int mp_classify(const mp_geometry* g, uint8_t* cls, int64_t* n_fluid, int64_t* n_interface,
                int64_t* n_cluster, void* stream);

/*
 * mp_step_noalloc -- one moment-propagation + sorption step of one propagated field of one
 * species, on caller-owned dense device arrays, that allocates no memory of any kind (no
 * cudaMalloc, no cudaFree, no allocating library routine). It serves callers that cannot
 * allocate device memory themselves or let a library do so: code running inside a host
 * application that owns every device allocation (a fixed budget or its own memory pool),
 * or code that must avoid the implicit device synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart; the update is the same as mp_step's (same readings, same
 * rounding of link probabilities), recomputed from the solid mask and u on every call.
 *
 *  nx, ny, nz    lattice (each >= 3); N = nx*ny*nz must not exceed 2,097,152 nodes: the
 *                step's FP64 reduction uses a fixed scratch array of 8192 block partials
 *                (64 KiB plus a counter, a __device__ array that every GPU using this entry
 *                point keeps until the library is unloaded). Larger N returns MP_EINVAL.
 *  solid         device, N bytes, nonzero = solid.
 *  u             device, FP32 3*N SoA, or NULL (rest).
 *  D_b, k_a, k_d as for mp_init.
 *  direction     0, 1, 2: Z_out = sum_r X_out(r) u*_g(r) (the VACF term of a velocity
 *                moment); -1: Z_out = sum_r X_out(r) (the free mass).
 *  X, X_ads      device, FP32, N each: the field and its adsorbed partner (dense; X_ads is
 *                read on interfacial nodes only).
 *  X_out, X_ads_out  device, FP32, N each, written everywhere (zero on solid nodes, X_ads_out
 *                zero off the interface); no byte of either may lie in X, X_ads, solid, u,
 *                Z_out or the other output (MP_EINVAL otherwise).
 *  Z_out         device, one double, written when the step completes.
 *  stream        cudaStream_t or NULL. Asynchronous.
 * The first call on a device looks up the scratch array's device address (with that device
 * current) and remembers it with the id of the device's context; make that first call before
 * any stream capture. After a cudaDeviceReset the next call finds a new context and looks the
 * address up again (so it is again a first call). Every call shares the
 * one scratch array and leaves its contents behind: the counter is cleared by each call, so
 * calls that overlap on the GPU (different streams, concurrent host threads) race and must
 * be serialised by the caller.
 * Errors: MP_EINVAL, MP_ECUDA.
 */
int mp_step_noalloc(int nx, int ny, int nz, const uint8_t* solid, const float* u, double D_b,
                    double k_a, double k_d, int direction, const float* X, const float* X_ads,
                    float* X_out, float* X_ads_out, double* Z_out, void* stream);

/*
 * mp_variant -- text naming how mp_step runs the context (no counterpart in the paper):
 * "flux" for MP_SCHEME_FLUX; for MP_SCHEME_DIRECT the launch form ("per-step" or
 * "persistent"), the link terms ("table" or "recompute") and the block size. Valid until the
 * context is freed.
 *
 * A persistent launch runs many steps with a device-wide barrier between them. Every wait
 * at that barrier is bounded (2 s); a wait that gives up makes the launch return early, and
 * the next call that synchronises the context (mp_vacf, mp_mass, mp_get_field) fails with
 * MP_ETIMEOUT: the fields and series written after the failed step are then not valid.
 */
const char* mp_variant(mp_ctx* c);

/*
 * mp_grid_wait_selftest -- runs the bounded device-wide barrier of the persistent step on its
 * own (no counterpart in the paper): n_blocks co-resident blocks of 32 threads meet at
 * `rounds` barriers. With `unreachable` nonzero every barrier waits for one block more than
 * the grid holds (an arrival that never comes), so each wait must give up after timeout_ns
 * nanoseconds; the call then returns MP_ETIMEOUT and the device stays usable.
 *  stream   cudaStream_t or NULL; synchronised before return.
 * Errors: MP_EINVAL (more blocks than can be resident at once, rounds outside 1..1e6,
 * timeout_ns outside 0..1e10), MP_ECUDA, MP_ETIMEOUT.
 */
int mp_grid_wait_selftest(int n_blocks, int rounds, int unreachable, int64_t timeout_ns, void* stream);

/* mp_free -- release a context and all its device memory (NULL is accepted). */
void mp_free(mp_ctx* c);

/* Text of the calling thread's last failure ("" if none); valid until its next call. */
const char* mp_last_error(void);

/*
 * lb_steady -- steady BGK lattice-Boltzmann flow through a medium.
 *
 * Paper: Eq. (lb_evolution), f_i(r + c_i dt, t + dt) = f_i(r,t) + Delta_i(r,t), with a BGK
 * collision Delta_i = -(f_i - f_i^eq)/tau, the Guo body-force term for a uniform force F on
 * fluid nodes, u = (sum_i f_i c_i + F/2)/rho, and halfway bounce-back on links into solid
 * nodes. Populations are stored in FP32 as deviations f_i - w_i; the residual is FP64.
 * The force acts on the largest connected fluid cluster only (see mp_classify): a uniform
 * force in a sealed pocket is balanced by pressure, so its steady velocity is zero there.
 *
 *  g             the medium (host or device mask; copied for the call).
 *  force         host, 3 doubles: body force per node.
 *  tau           relaxation time, > 1/2.
 *  tol           stop at the first checked step t with max |u(t) - u(t-1)| < tol, taken
 *                over fluid nodes and components.
 *  max_steps     step budget (>= 1); check_every: residual period (>= 1); the residual is
 *                also taken at t = max_steps. After every check that fails (before
 *                max_steps) the populations are replaced by the mean of the last two
 *                iterates: this keeps the fixed point and removes the undamped period-2
 *                modes that bounce-back sustains at nodes with few open links.
 *  u_init        device, FP32 3*N, or NULL (rest): starting velocity;
 *  rho_init      device, FP32 N, or NULL (1 everywhere): starting density. The start is
 *                f^eq(rho_init, u_init); NULL, NULL is the cold start from rest. The mass of
 *                every connected fluid region is conserved from the start, so a warm start
 *                reaches the cold start's steady state only with the same mass per region.
 *  u_out         device, FP32 3*N: u at the final step, zero on solid nodes.
 *  rho_out       device, FP32 N, or NULL: the density at the final step (0 on solids).
 *  steps_out, residual_out   host (either may be NULL): steps taken, last residual.
 *  stream        cudaStream_t or NULL. Allocates its working populations stream-ordered
 *                and frees them before returning; synchronises the stream.
 * Returns MP_OK when converged, MP_ENOTCONVERGED when max_steps ran out or the velocity
 * became non-finite (an unstable run stops at that check with residual_out = +inf; u_out,
 * steps_out and residual_out are still written), MP_EINVAL, MP_ENOMEM or MP_ECUDA.
 */
int lb_steady(const mp_geometry* g, const double force[3], double tau, double tol,
              int64_t max_steps, int64_t check_every, const float* u_init, const float* rho_init,
              float* u_out, float* rho_out, int64_t* steps_out, double* residual_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MP_H */
