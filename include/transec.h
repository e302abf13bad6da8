/*
 * transec.h -- C ABI of the GB300 library for CAP-terminated Landauer transmission.
 *
 * The library computes, on one GPU, the k-resolved transmission of a real-space
 * finite-difference Kohn-Sham Hamiltonian with lateral periodic boundaries and
 * complex absorbing potentials (CAPs) at the two transport ends, following
 * Zhu, Feldman & Dunham, arXiv 2208.02783 ("Highly parallelizable electronic
 * transport calculations in periodic Rhodium and Copper nanostructures"):
 *
 *   G(E, k)  = [E - H_k + i(Gamma_L + Gamma_R)]^-1          (Sec. II.A)
 *   T(E, k)  = 4 Tr[Gamma_L G^dagger Gamma_R G]             (Sec. II.A; the factor 4
 *              goes with Gamma entering G as i*Gamma, so that T counts open channels)
 *            = sum_{j : Gamma_L(j) > 0} t_j,
 *   t_j      = 4 Gamma_L(j) sum_i Gamma_R(i) |x_j(i)|^2,    A(E, k) x_j = e_j
 *   T(E)     = sum_k w_k T(E, k)                            (Sec. II.A, k-averaging)
 *
 * H_k (Sec. II.A, Eqs. Bloch and H_k) is -1/2 times the order-2N central
 * finite-difference Laplacian plus the local potential V_KS, on a uniform grid with
 * index n = i + nx*(j + ny*l); a lateral neighbour that leaves the cell re-enters on
 * the other side with the Bloch factor exp(i k_a L_a w) (w = number of wraps), and
 * z has zero Dirichlet ends.  The columns x_j are found with Krylov methods: COCG
 * when H_k is real (kappa in {0, 1/2} on both axes, A complex symmetric), otherwise
 * BiCG with the transposed shadow system -- the conjugate-orthogonal CG of the
 * complex symmetric +-k operator of Sec. II.B (Eq. def-Gk) -- which also returns
 * the columns of A(E, -k) = A(E, k)^T, hence T(E, -k), in the same run.
 *
 * Conventions for every entry point:
 *   - Units are Hartree and bohr.  T is per spin (Sec. III).
 *   - Host pointers unless stated; inputs are copied, never retained.
 *   - The caller owns every output buffer.
 *   - Each call returns a transec_status; on failure transec_last_error() describes
 *     it.  No call traps or aborts: GPU-side failures come back as status codes.
 *   - A context is not thread-safe; use one per host thread.  Work is queued on the
 *     context's stream and every call below returns after its results are written.
 */
#ifndef TRANSEC_H
#define TRANSEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct transec_ctx transec_ctx;

/* Status codes.  Per-result codes use the same values. */
enum transec_status {
  TRANSEC_OK = 0,
  TRANSEC_EINVAL = -1,     /* bad argument (size, order, pointer, NaN input) */
  TRANSEC_ENOMEM = -2,     /* device or host allocation failed */
  TRANSEC_ECUDA = -3,      /* a CUDA call failed; see transec_last_error */
  TRANSEC_ENOCONV = -4,    /* a column hit maxit before the tolerance; its t is NaN */
  TRANSEC_EBREAKDOWN = -5, /* Krylov breakdown (zero or non-finite scalar); t is NaN */
  TRANSEC_ETIMEOUT = -6,   /* a bounded device wait gave up */
  TRANSEC_ESTATE = -7      /* call order violated (e.g. no potential set yet) */
};

/* Krylov method. */
enum transec_method {
  TRANSEC_METHOD_AUTO = 0, /* COCG where H_k is real, transpose BiCG elsewhere */
  TRANSEC_METHOD_COCG = 1, /* only valid where H_k is real */
  TRANSEC_METHOD_BICG = 2  /* transpose BiCG (+-k pair) everywhere */
};

/* Arithmetic of the iteration. */
enum transec_precision {
  TRANSEC_PREC_FP64 = 0,  /* complex128 vectors and stencil throughout */
  TRANSEC_PREC_MIXED = 1, /* complex64 vectors and stencil with FP64 scalars, FP64
                             solution accumulation and FP64 residual replacement */
  TRANSEC_PREC_DF64 = 2   /* multi-shift engine only (transec_shifted_columns,
                             transec_transmission_sketch): vectors stored and the stencil,
                             vector and per-shift updates computed in double-float (pairs
                             of floats, ~2^-47 relative rounding) on the FP32 pipes, Krylov
                             scalars in FP64; the other solvers run it as FP64 */
};

typedef struct transec_solver_opts {
  int method;         /* enum transec_method (default AUTO) */
  int precision;      /* enum transec_precision (default FP64) */
  double tol;         /* per column: ||A x - e_j||_2 <= tol (||e_j|| = 1); default 1e-10;
                         BiCG requires the shadow residual to meet it too */
  int maxit;          /* operator applications per half and column; default 100000 */
  int slots;          /* columns in flight on the GPU; 0 = chosen by the autotuner */
  int chunk;          /* iterations per graph launch between host polls; 0 = default */
  double reliable;    /* mixed precision: fold the FP32 correction into the FP64
                         solution, recompute the FP64 residual and restart the FP32
                         iteration once its residual has dropped by this factor (or
                         has stalled); default 1e-5 */
  int tile_y;         /* stencil tile rows (0 = autotune); tiles span min(nx, 32) */
  int slab;           /* most z-planes per stencil block; the depth used splits nz into equal slabs (0 = default) */
  int profile;        /* != 0: time every stencil and update launch with CUDA events on
                         the context's stream (read back with transec_stats) */
  int mixed_maxit;    /* mixed precision: FP32 iterations a column may take before it is
                         handed to the plain FP64 engine (solved again from scratch);
                         default 8000 */
  int mixed_decade_its; /* mixed precision: a column whose FP32 residual has fallen by less
                         than one decade per this many iterations (checked from that many
                         iterations on) is handed to the FP64 engine; default 1000,
                         negative = never */
  int host_loop;      /* 0 (default): the whole solve is one CUDA-graph launch whose
                         device-side WHILE loop runs chunk after chunk until the queue is
                         drained (bounded by maxit); != 0: the host launches and polls one
                         chunk graph at a time (always the case when profile != 0) */
  int df_stall_its;   /* double-float multi-shift runs: once a run has gone this many
                         iterations without a new shift converging (counted from its
                         first convergence, or 3x this from the start), its remaining
                         shifts stop and are solved again in FP64; default 8000,
                         negative = never */
  int psym;           /* != 0: transec_transmission_sketch runs P-symmetric COCG instead
                         of transpose BiCG (Sec. II.C: with V invariant under the in-plane
                         rotation R_{z,pi} about grid point (0, 0), A(E, k)^T = P_k A(E, k)
                         P_k^-1 for the Bloch-phased inversion P_k, so one operator
                         application per iteration serves both k and -k).  Requires
                         precision = TRANSEC_PREC_DF64, a potential that passes the
                         inversion check of transec_set_potential, nx <= 32 and
                         nx * ny <= 896; other entry points ignore it.  Default 0 */
  double sketch_guard; /* transec_transmission_sketch: a result whose sketch may miss more
                         of T than this (the missed-energy estimate of miss_out), or, with
                         transpose-BiCG runs, whose two independent estimates differ by
                         more, |T(E, k) - T(E, -k)| > sketch_guard, is computed again with
                         a sketch of twice the sizes (up to 32 + 64) and a fresh draw, up
                         to three times; default 1e-7 (a tenth of the 1e-6 bar on T),
                         negative = never */
} transec_solver_opts;

/* Library version (major*10000 + minor*100 + patch). */
int transec_version(void);

/* Human-readable name of a status code (static storage). */
const char* transec_status_string(int status);

/*
 * Create a context for an nx x ny x nz grid with spacings hx, hy, hz (bohr) and a
 * finite-difference Laplacian of order fd_order in {2, 4, ..., 12} (Sec. I: the
 * real-space grid Hamiltonian of PARSEC/TRANSEC).  device is a CUDA ordinal;
 * cuda_stream is a cudaStream_t to order work after (NULL = the legacy default
 * stream).  *out receives the context, or NULL on failure.
 * Errors: EINVAL (sizes < 1, nz < 2, order not even in [2, 12], h <= 0),
 *         ECUDA, ENOMEM.
 */
int transec_create(transec_ctx** out, int nx, int ny, int nz, double hx, double hy,
                   double hz, int fd_order, int device, void* cuda_stream);

/*
 * Set the local Kohn-Sham potential V_KS (Sec. II.A, Eq. H_k), nx*ny*nz doubles in
 * grid order (x fastest), Hartree.  on_device != 0 means v_ks is a device pointer
 * on the context's device.  Errors: EINVAL (NULL, non-finite value), ECUDA.
 */
int transec_set_potential(transec_ctx* ctx, const double* v_ks, int on_device);

/*
 * Set the absorbing profiles Gamma_L(z), Gamma_R(z) (Sec. II.A, Eq. CAP-Gaussian:
 * constant in the xy-plane, so one value per z-plane), nz doubles each, Hartree,
 * host memory.  The left-CAP support {j : Gamma_L(plane(j)) > 0}, ordered by grid
 * index, defines the right-hand sides e_j; its size is transec_n_rhs().
 * Errors: EINVAL (NULL, negative or non-finite value, empty left support).
 */
int transec_set_abc(transec_ctx* ctx, const double* gamma_l, const double* gamma_r);

/*
 * Set the lateral k-mesh (Sec. II.A: T(E) is the average of T_k(E) over sampled k).
 * kfrac holds nk pairs (k_a L_a / 2pi, k_b L_b / 2pi); weights holds nk values
 * (NULL = uniform 1/nk).  Host memory.  Errors: EINVAL (nk < 1, non-finite).
 */
int transec_set_kmesh(transec_ctx* ctx, int nk, const double* kfrac, const double* weights);

/* Replace / read the solver options (fields left 0 take their defaults). */
int transec_set_solver(transec_ctx* ctx, const transec_solver_opts* opts);
int transec_get_solver(const transec_ctx* ctx, transec_solver_opts* opts);

/*
 * Autotune the launch shape for this context's operator (no counterpart in the
 * paper: a property of the GPU kernels).  For each candidate stencil tile height,
 * z-slab depth and number of columns in flight it runs a bounded burst of Krylov
 * iterations (maxit 32) at energy E and k index ik in the configured precision,
 * measures the stencil and update kernels with CUDA events, and keeps the candidate
 * with the most point-applications per second in the solver options (tile_y, slab,
 * slots).  The chosen values are also written to the non-NULL outputs.  Counters
 * (transec_stats) are reset afterwards.  Errors: as transec_column_contributions.
 */
int transec_autotune(transec_ctx* ctx, double energy, int ik, int* tile_y_out, int* slab_out,
                     int* slots_out);

/* Number of left-CAP columns (right-hand sides per (E, k)). */
int transec_n_rhs(const transec_ctx* ctx, int64_t* n_rhs);

/*
 * Full transmission: for every energy energies[e] (Hartree) and every k of the mesh,
 * solve all left-CAP columns and write T_out[e*nk + k] = T(E_e, k).  If T_avg_out is
 * not NULL it receives T(E_e) = sum_k w_k T(E_e, k).  status_out (ne*nk ints, may be
 * NULL) receives the worst status over that (E, k)'s columns; iters_out (ne*nk ints,
 * may be NULL) the largest iteration count.  With BiCG, a k whose mirror -k is also
 * in the mesh is not solved again: T(E, -k) comes from the shadow columns of k.
 * An (E, k) with a failed column gets T = NaN; the call then returns the most
 * severe status and every other result stays valid.  Host memory.
 */
int transec_transmission(transec_ctx* ctx, int ne, const double* energies, double* T_out,
                         double* T_avg_out, int* status_out, int* iters_out);

/*
 * Sampled columns: for item i, solve A(energies[i], k_{ik[i]}) x = e_j with j the
 * cols[i]-th left-CAP column (0 <= cols[i] < n_rhs) and write t_out[i] = t_j.  If
 * t_minus_out is not NULL it receives t_j at (E, -k) (from the BiCG shadow column;
 * equal to t_out where H_k is real).  iters_out / status_out (may be NULL) receive
 * per-item iteration counts and statuses.  With on_device != 0 every array argument
 * is a device pointer on the context's device (energies double, ik int32, cols int64,
 * outputs double / int32); otherwise host memory.  Returns the most severe status.
 */
int transec_column_contributions(transec_ctx* ctx, int nitems, const double* energies,
                                 const int* ik, const int64_t* cols, double* t_out,
                                 double* t_minus_out, int* iters_out, int* status_out,
                                 int on_device);

/*
 * Batched sampled columns over several operators: item i is a column of context
 * ctxs[ictx[i]] (a cell of its own size, potential, CAPs and k-mesh), solved at energy
 * energies[i] and k index ik[i] of that context's mesh, column cols[i] of its left-CAP
 * support; outputs as in transec_column_contributions.  The paper computes each
 * (k, spin) independently on separate nodes (Appendix); here independent operators
 * of uneven size share one slot engine, so one solve keeps the GPU full across all of
 * them.  Every context must be ready, live on the same device and use the same
 * stencil order; the solve runs with ctxs[0]'s solver options, buffers and stream.
 * With on_device != 0 every array is a device pointer (ictx int32).  Returns the most
 * severe per-item status; EINVAL for mismatched contexts or an out-of-range ictx / ik.
 */
int transec_batch_column_contributions(int nctx, transec_ctx* const* ctxs, int nitems,
                                       const int* ictx, const double* energies, const int* ik,
                                       const int64_t* cols, double* t_out, double* t_minus_out,
                                       int* iters_out, int* status_out, int on_device);

/*
 * Operator apply (the hot-path stencil on its own): y_v = A(E, k_ik) x_v for nvec
 * vectors of nx*ny*nz complex128 values (interleaved re, im; grid order), stored
 * one after another.  conj_k != 0 applies A(E, -k) = A(E, k)^T instead.  Device
 * pointers (on_device != 0) or host memory.  Used to check the stencil on its own.
 */
int transec_apply(transec_ctx* ctx, double energy, int ik, int conj_k, int nvec,
                  const double* x, double* y, int on_device);

/*
 * Operator apply that allocates nothing (the paper has no counterpart: this is a
 * library service).  For callers that may not have the library call cudaMalloc or
 * cudaFree -- a process whose device memory is owned by another allocator, or a
 * latency-critical loop that cannot take cudaFree's implicit synchronisation --
 * this computes the same y_v = A(E, k_ik) x_v (A(E, -k) if conj_k != 0) as
 * transec_apply, for nvec complex128 vectors in grid order, with x and y DEVICE
 * pointers on the context's device.  The stencil's scratch lives in a fixed static
 * device array of about 17 MiB that every GPU loading the library holds until exit;
 * limits: nvec <= 64 and nvec * nx * ny * nz <= 1048576 (EINVAL beyond them, with a
 * message naming the limit).  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call before
 * any stream capture.  All calls share the array: calls that overlap on the GPU
 * race, so issue them one after another.  The context itself is created (and its
 * buffers allocated) beforehand by transec_create / transec_set_*.
 */
int transec_apply_noalloc(transec_ctx* ctx, double energy, int ik, int conj_k, int nvec,
                          const double* x, double* y);

/*
 * Column trace (the reduction on its own): for nvec solution vectors x_v (complex128,
 * grid order, one after another) and left-CAP column positions cols[v], write
 * t_out[v] = 4 Gamma_L(j_v) sum_i Gamma_R(i) |x_v(i)|^2.  Device or host memory.
 */
int transec_trace(transec_ctx* ctx, int nvec, const double* x, const int64_t* cols,
                  double* t_out, int on_device);

/*
 * Counters of the solves since the last transec_stats_reset (or creation):
 * launches = library kernels launched; point_applies = operator applications summed
 * over columns and halves, times grid points (the work the stencil did); with
 * opts.profile set, stencil_ms / update_ms = summed device time of the stencil and
 * vector-update launches and stencil_launches / update_launches their counts;
 * fallbacks = mixed-precision columns that did not converge in the mixed form and
 * were solved again by the plain FP64 engine.  point_applies / stencil_ms /
 * stencil_launches count the FP64 kernels; point_applies32 / stencil32_ms /
 * stencil32_launches the FP32 kernels of the mixed form.  Any output may be NULL.
 */
int transec_stats(const transec_ctx* ctx, long long* launches, long long* point_applies,
                  double* stencil_ms, long long* stencil_launches, double* update_ms,
                  long long* update_launches, long long* fallbacks, long long* point_applies32,
                  double* stencil32_ms, long long* stencil32_launches);
int transec_stats_reset(transec_ctx* ctx);

/*
 * Learned right preconditioner (an extension; the paper has no learned component): a
 * 3D U-Net with 3 levels of 16/32/64 channels, 3x3x3 convolutions (zero padding),
 * ReLU, 2x2x2 average pooling, nearest 2x upsampling and skip concatenation, 4 input
 * channels (Re r, Im r, V, Gamma) and 2 outputs (Re e, Im e).  Its convolutions run as
 * BF16 tensor-core implicit GEMMs with FP32 accumulation (forward, data gradient,
 * weight gradient), trained with Adam on FP32 master weights.  The forward and
 * data-gradient convolutions use tcgen05 MMAs with the accumulator in tensor memory
 * when a lateral plane of the level (with a one-voxel halo) fits the block's shared
 * memory, mma.sync tiles otherwise; the weight gradient uses mma.sync.  A network is
 * built for one volume nx x ny x nz (each a multiple of 4).
 */
typedef struct transec_unet transec_unet;

/* Create a network with He-initialised weights from `seed`.  Errors: EINVAL (sizes),
 * ENOMEM, ECUDA. */
int transec_unet_create(transec_unet** out, int device, int nx, int ny, int nz,
                        unsigned long long seed);
/* Parameter count and flat FP32 parameters in host memory: per layer (e1a, e1b, e2a,
 * e2b, e3a, e3b, d2a, d2b, d1a, d1b, out) the weights (27, cout, cin) then the bias
 * (cout).  set_params(NULL) only resets the optimiser state. */
int transec_unet_n_params(const transec_unet* u, long long* n);
int transec_unet_set_params(transec_unet* u, const float* params);
/* Zero the output layer's weights (its bias is kept) and reset the optimiser state: the
 * learned preconditioner's starting point (the first Adam steps then learn a
 * correlation with the target instead of shrinking a random output of the wrong
 * scale).  Errors: EINVAL, ECUDA. */
int transec_unet_zero_output(transec_unet* u);
int transec_unet_get_params(transec_unet* u, float* params);
/* out[v][0..1] = network(in[v][0..3]) for every voxel v = x + nx(y + ny z); FP32, device
 * (on_device != 0) or host memory. */
int transec_unet_forward(transec_unet* u, const float* in, float* out, int on_device);
/* One training step on one volume: relative loss sum|y - t|^2 / sum|t|^2 against
 * target[v][0..1], backward, and an Adam update when lr > 0.  loss / grads (host, flat
 * layout) may be NULL.  Device or host arrays.  forward and train_step return
 * ETIMEOUT when a tcgen05 convolution gave up waiting for its MMAs (bounded wait). */
int transec_unet_train_step(transec_unet* u, const float* in, const float* target, float lr,
                            float* loss, float* grads, int on_device);
/* Convolution kernels: 0 (default) tcgen05 where the plane fits, else mma.sync; 1 the
 * mma.sync kernels only.  Errors: EINVAL. */
int transec_unet_set_path(transec_unet* u, int path);
/* One 3x3x3 convolution of the network alone (zero padding), on `device`:
 * y[v][o] = b[o] + sum over taps t and input channels i of w[t][o][i] x[v + d_t][i],
 * tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), voxel v = x + nx(y + ny z).  x: [nx*ny*nz][cin]
 * and w: [27][cout][cin] as bfloat16 bit patterns, b: [cout] float (may be NULL), y:
 * [nx*ny*nz][cout] float; host arrays, FP32 accumulation.  path 0: the tcgen05 kernel
 * where the plane fits (else mma.sync), 1: the mma.sync kernel.  cin, cout multiples of
 * 16 (cout <= 256).  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
int transec_unet_conv3d(int device, int nx, int ny, int nz, int cin, int cout, const uint16_t* x,
                        const uint16_t* w, const float* b, float* y, int path);
/* Volume the network was built for.  Any output may be NULL. */
int transec_unet_dims(const transec_unet* u, int* nx, int* ny, int* nz);
const char* transec_unet_last_error(const transec_unet* u);

/*
 * Fit the network to the operator family A(E, k) = E - H_k + i Gamma of `ctx`
 * (Sec. II.A; same volume): `steps` Adam steps
 * at learning rate lr, each on one pair (r, e) with r = A(E, k) e, E uniform in
 * [e_lo, e_hi] and k uniform over the mesh, all drawn from `seed`.  source 0: e is a
 * seeded random complex field (standard normals smoothed by 0, 1, 2, 3, 5 or 8 passes
 * of a [1 2 1]/4 filter per axis; periodic in x and y, zero outside in z).  source 1:
 * e = x* - x_i for up to 48 iterates x_i (x_0 = 0 included) of a transpose-BiCG solve
 * of a random left-CAP column at opts.tol / opts.maxit, x* its solution; the pairs of
 * one column are used once each, in random order, before the next column is drawn.
 * The network input is (s_r Re r, s_r Im r, V - E, Gamma) and the target s_e e, with
 * s_r = sqrt(n) / ||r|| and s_e = sqrt(n) / ||e||.  loss_out (host, `steps` floats,
 * may be NULL) receives each step's relative loss.  Errors: EINVAL (arguments, volume
 * mismatch), ESTATE, ENOMEM, ECUDA; ENOCONV / EBREAKDOWN when the column solves of
 * source 1 keep failing.
 */
int transec_unet_train_operator(transec_ctx* ctx, transec_unet* net, int source, int steps,
                                double e_lo, double e_hi, float lr, unsigned long long seed,
                                float* loss_out);

/*
 * Sampled columns by FGMRES(restart) with the network as right preconditioner on every
 * net_every-th Arnoldi step (1: every step; 2: alternating with the identity) and the
 * identity on the others; net == NULL gives plain restarted GMRES.  Item i solves
 * A(energies[i], k_{ik[i]}) x = e_j for the cols[i]-th left-CAP column to
 * ||e_j - A x|| <= opts.tol in FP64 and writes t_out[i] = t_j, the column's share of
 * T(E, k) (Sec. II.A; the same quantity as transec_column_contributions).  A column whose residual
 * has not halved over 10 restart cycles, that reaches maxit operator applications, or
 * whose Hessenberg matrix turns singular (a zero preconditioned direction) is solved
 * again by the plain FP64 Krylov engine (fallback_out[i] = 1).  iters_out
 * receives the operator applications of both.  Host arrays; returns the most severe
 * item status (failed items get t = NaN).  Errors: EINVAL, ESTATE, ENOMEM, ECUDA.
 */
int transec_fgmres_columns(transec_ctx* ctx, transec_unet* net, int net_every, int nitems,
                           const double* energies, const int* ik, const int64_t* cols,
                           int restart, int maxit, double* t_out, int* iters_out,
                           int* status_out, int* fallback_out);
void transec_unet_destroy(transec_unet* u);

/*
 * One left-CAP column at ne energies by a multi-shift transpose BiCG: A(E, k) differs
 * from A(E0, k) by (E - E0) times the identity (Sec. II.A), so one Krylov run seeded at
 * the middle energy E0 yields every energy's column through collinear residuals, with
 * the per-energy iterates kept on the Gamma_R planes the trace reads.  Writes
 * t_out[s] = t_j and, if not NULL, t_minus_out[s] = t_j at -k (from the shadow system,
 * Sec. II.B) for energies[s]; iters_out[s] = seed iterations at which energy s
 * converged (||e_j - A x|| <= opts.tol, from the seed residual); status_out[s] its
 * status.  Host arrays; 1 <= ne <= 4096.  A host-driven single-column form of the
 * method.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA; per-energy ENOCONV / EBREAKDOWN.
 */
int transec_shifted_column(transec_ctx* ctx, int ne, const double* energies, int ik, int64_t col,
                           double* t_out, double* t_minus_out, int* iters_out, int* status_out);

/*
 * Sampled columns at a whole window of energies by the multi-shift engine (the slot
 * engine of transec_column_contributions with every run serving ne energies):
 * A(E, k) = A(E0, k) + (E - E0) 1 (Sec. II.A), so one transpose-BiCG run seeded at the
 * middle energy E0 of the window yields every energy's column of G(E, k) e_j and, from
 * its shadow system, of G(E, -k) e_j (A(E, k)^T = A(E, -k), Sec. II.B).  The per-energy
 * iterates are kept only on the Gamma_R planes the trace reads.  Item i is the
 * cols[i]-th left-CAP column at k index ik[i]; for every energy s it writes
 * t_out[i*ne + s] = t_j(E_s, k), t_minus_out[i*ne + s] = t_j(E_s, -k) (may be NULL),
 * iters_out[i*ne + s] = seed iterations at which energy s converged
 * (||e_j - A(E_s) x|| <= opts.tol, from the collinear seed residual) and
 * status_out[i*ne + s] (may be NULL).  Runs retire and refill on the GPU as in the
 * plain engine (opts.slots runs in flight, 0 = chosen from the grid size and free
 * memory); the whole solve is one graph launch with a device-side loop unless
 * opts.profile or opts.host_loop is set.  With opts.precision = TRANSEC_PREC_DF64 the
 * runs are double-float, and the (item, energy) results that do not converge that way
 * (or stop under opts.df_stall_its) are solved again in FP64 within the call.  Host
 * arrays; 1 <= ne <= 1024.  Failed (E, item) results get t = NaN and the call returns
 * the most severe status.  Errors: EINVAL, ESTATE, ENOMEM, ECUDA, ETIMEOUT.
 */
int transec_shifted_columns(transec_ctx* ctx, int ne, const double* energies, int nitems,
                            const int* ik, const int64_t* cols, double* t_out, double* t_minus_out,
                            int* iters_out, int* status_out);

/*
 * Full-trace transmission T(E, k) and T(E, -k) for a window of energies from a
 * two-sided randomized sketch of M = Gamma_R^1/2 G Gamma_L^1/2 (Sec. II.A:
 * T = 4 Tr[Gamma_L G^dagger Gamma_R G] = 4 ||M||_F^2).  M has numerical rank about the
 * number of open (and barely closed) channels at (E, k) (Sec. III), far below its
 * n_rhs columns, so instead of n_rhs unit columns the library solves, for each k of
 * ik[0..nrep-1], s_left runs with random right-hand sides Gamma_L^1/2 omega and s_right
 * runs with Gamma_R^1/2 psi (omega, psi: unit-modulus random phases from `seed`, by
 * splitmix64), every run a multi-shift transpose BiCG over the whole window (as in
 * transec_shifted_columns).  The LEFT runs give Y = M Omega, the RIGHT runs' shadow
 * systems W = Psi^T M (and the other halves the same pair at -k); per energy and
 * sign of k the library forms Q = orth(Y), X = (Psi^T Q)^+ W and T = 4 ||X||_F^2 (the
 * two-sided low-rank approximation of Tropp, Yurtsever, Udell & Cevher, SIAM J. Matrix
 * Anal. Appl. 2017), exact to rounding when the numerical rank of M is at most s_left.
 * T_out[r*ne + s] = T(E_s, k_{ik[r]}); T_minus_out[r*ne + s] = T(E_s, -k) computed from
 * the other halves (equal to T(E_s, k) in exact arithmetic, Sec. II.B: an independent
 * estimate, so |T - T_minus| gauges the sketch error); rank_out = directions of Y kept;
 * status_out per result; iters_out = seed iterations at which the energy converged in
 * its slowest run.  1 <= s_left <= 32, s_left <= s_right <= 64, 1 <= ne <= 1024.  All
 * nrep * (s_left + s_right) runs are in flight at once (no refill).  With
 * opts.precision = TRANSEC_PREC_DF64 the runs are double-float, and the (k, energy)
 * results that do not converge that way (or stop under opts.df_stall_its) are
 * computed again with FP64 runs within the call.  With opts.psym set the runs are
 * P-symmetric COCG (one half each): Y and W at +k come from the primal solutions and
 * their images under P_k (test vectors P_k psi for W), the -k pair from the same data
 * mirrored, so T_minus equals T to rounding and is no independent estimate; EINVAL
 * when opts.psym is set with another precision, a potential that is not
 * inversion-symmetric (relative gap above 1e-12) or a plane too large for one tile.
 * The FP64 re-solve of failed results uses transpose BiCG.  miss_out (may be NULL) =
 * 4 ||(1 - P) y||^2 for the last LEFT run's column y = M omega and P the projector on
 * the span of the other LEFT columns: since E ||(1 - P) M omega||^2 = ||(1 - P) M||_F^2
 * for unit-modulus omega, it estimates the part of T = 4 ||M||_F^2 outside the span of
 * s_left - 1 random directions (the larger of the two signs of k).  Results with
 * miss_out above opts.sketch_guard, or (without opts.psym) with T and T_minus apart by
 * more, are computed again with a doubled sketch (the a-posteriori checks acting);
 * rank_out, miss_out then report the larger sketch and iters_out adds its
 * iterations.  Host arrays.
 * Errors: EINVAL, ESTATE, ENOMEM, ECUDA, ETIMEOUT; per-result ENOCONV / EBREAKDOWN with
 * T = NaN.
 */
int transec_transmission_sketch(transec_ctx* ctx, int ne, const double* energies, int nrep,
                                const int* ik, int s_left, int s_right, unsigned long long seed,
                                double* T_out, double* T_minus_out, int* rank_out, int* status_out,
                                int* iters_out, double* miss_out);

/*
 * The paper's eigen route, its per-energy stage (Sec. II.A, Eqs.
 * transmission-eigenbasis, Gamma-tilde, G-diag; Sec. II.B; Sec. II.D's truncation to a
 * fraction of the eigenpairs): T(E, k) from p eigenpairs of B(k) = H_k - i Gamma,
 *   T(E) = 4 sum_{m,n} conj(g_m) g_n Rt[m, n] Lt[n, m],  g_n = 1/(E - lambda_n),
 *   Rt = V^H Gamma_R V,  Lt = W^T Gamma_L conj(W),
 * with V the right eigenvectors and W the left ones (W^T B = diag(lambda) W^T),
 * normalised so that W^T V = 1 on the full grid (W are the right eigenvectors of
 * B(-k)).  The caller supplies the eigensolution (the library does not compute it):
 * lambda [p] complex (interleaved re, im); v_right [n_R][p] complex, the rows of V on
 * the right-CAP support and w_left [n_L][p] complex, the rows of W on the left-CAP
 * support, each support in grid order (the planes with Gamma > 0 ascending, x fastest
 * within a plane; n_R = right-CAP planes x nx ny).  With every eigenpair the result is
 * the exact T(E, k); with the p nearest the energies it is the paper's truncated sum.
 * T_out [ne].  Host arrays; 1 <= p <= 10240.  Errors: EINVAL, ESTATE (CAPs not set),
 * ENOMEM, ECUDA.
 */
int transec_eigen_transmission(transec_ctx* ctx, int p, const double* lambda, const double* v_right,
                               const double* w_left, int ne, const double* energies, double* T_out);
/* With opts.profile set, the event-timed ms since the last transec_stats_reset of the
 * eigen route's two Gram-matrix launches and of its eigen-sum launch.  Either output
 * may be NULL. */
int transec_eigen_stats(const transec_ctx* ctx, double* gram_ms, double* sum_ms);

/*
 * Counters of the multi-shift engine since the last transec_stats_reset: seed
 * iterations summed over runs, per-shift point updates (kept points x halves x
 * iterations of each shift), with opts.profile set the event-timed stencil and
 * shifted-update kernels (ms, launches) of the FP64 runs and, apart, of the
 * double-float runs (the *_df outputs), and the sketch reduction (ms), and the
 * (energy, column or k) results of double-float calls that were solved again in FP64
 * (fp64_redone), and the (energy, k) results of sketch calls computed again with a
 * larger sketch under opts.sketch_guard (guard_redone).  Any output may be NULL.
 */
int transec_sweep_stats(const transec_ctx* ctx, long long* iters, long long* shift_points,
                        double* stencil_ms, long long* stencil_launches, double* shift_ms,
                        long long* shift_launches, double* stencil_df_ms, long long* stencil_df_launches,
                        double* shift_df_ms, long long* shift_df_launches, double* reduce_ms,
                        long long* fp64_redone, long long* guard_redone);

/* Message of the last failure on this context ("" if none).  Valid until the next
 * call on the same context. */
const char* transec_last_error(const transec_ctx* ctx);

/* Release the context and everything it allocated.  NULL is ignored. */
void transec_destroy(transec_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TRANSEC_H */
