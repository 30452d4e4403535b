/*
 * kpz.h -- C ABI of the GB300 octahedron KPZ lattice engine.
 *
 * Model (Kelling, Odor, Nagy, Schulz, Heinig, arXiv:1204.5072, Sec. 2.1):
 * an L x L periodic lattice of octahedron slopes sigma_x, sigma_y = +-1; a site
 * that is a local minimum of its four neighbours is raised by 2 with
 * probability p, a local maximum is lowered by 2 with probability q
 * (eq. rule). One Monte Carlo step (MCS) is L*L update attempts. Time is
 * advanced with the paper's decomposition (Sec. 3, 3.1): a dead-border tile
 * grid whose origin moves to a random site every sweep, and single-hit double
 * tiling of each 128 x 128 tile into 4 x 4 cells with four 2 x 2 quadrant sets.
 * The random numbers are counter-based Philox4x32-10 keyed by
 * (seed, sample, sweep, tile, cell row, round), so a run is a pure function of
 * (L, p, q, seed, sample, tile shape, number of sweeps).
 *
 * Conventions
 *   - All functions return kpz_status; no C++ exception crosses this boundary.
 *   - Host pointers are owned by the caller and only read or written during
 *     the call. Device memory is owned by the context unless the caller passes
 *     `dev_buf` in kpz_opts, in which case the caller keeps it alive until
 *     kpz_free and the library never frees it.
 *   - Work is queued on the context's stream (kpz_opts.stream, or the legacy
 *     default stream when NULL). Functions that return data to the host
 *     synchronise that stream; kpz_run does not.
 *   - A context is not thread-safe; distinct contexts are independent.
 *   - After KPZ_ECUDA the context is poisoned: every later call returns
 *     KPZ_ESTATE until kpz_free.
 *
 * Packed exchange format (kpz_slopes / kpz_set_slopes): row j (y) occupies
 * L/16 consecutive 32-bit words; site i (x) sits in word j*(L/16) + i/16 at bit
 * 2*(i%16) (sigma_x, 1 = +1) and bit 2*(i%16)+1 (sigma_y). The engine's own
 * HBM layout is different and is not part of the ABI: one bit per site,
 * (h >> 1) & 1, which with the fixed site parity h = i + j + h(0,0) (mod 2)
 * determines every slope; bit-sliced per 4 x 4 cell row.
 */
#ifndef KPZ_H
#define KPZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KPZ_OK = 0,
    KPZ_EINVAL = 1,   /* invalid argument; nothing was launched or changed    */
    KPZ_ENOMEM = 2,   /* device allocation failed or dev_buf too small        */
    KPZ_ECUDA = 3,    /* a CUDA call failed; the context is now poisoned      */
    KPZ_ETIMEOUT = 4, /* a bounded device-side wait gave up                   */
    KPZ_ESTATE = 5,   /* context poisoned by an earlier error                 */
    KPZ_ENODEV = 6,   /* no usable CUDA device                                */
    KPZ_ERANGE = 7,   /* size beyond the fixed scratch of kpz_roughness_static */
    KPZ_ECKPT = 8     /* checkpoint file unreadable, unwritable, truncated,
                         not a checkpoint, or its checksum does not match    */
} kpz_status;

typedef struct kpz_ctx kpz_ctx;

/* Options; a NULL pointer or zero fields select the defaults. */
typedef struct {
    uint32_t bx, by;      /* tile shape in sites: bx = 128; by = 128 or 256 (0 = 128).
                             The tile shape is part of the schedule (Sec. 3.1), so
                             different shapes give different (equally valid)
                             trajectories; 128 x 256 needs L >= 256               */
    uint32_t run;         /* tiles per work item: the resident warps take runs of
                             `run` tiles of one tile row from a queue (power of two
                             <= L/128; 0 = min(8, L/128) below L = 65536, L/4096
                             from there); execution only, it does not change the
                             result                                                */
    uint32_t warps_per_cta; /* 1..8; 0 = 4 for 128-row tiles from L = 65536, else 8;
                             execution only                                        */
    void* stream;         /* cudaStream_t to queue work on (NULL = default stream)  */
    void* dev_buf;        /* optional caller-owned device memory for the lattice and
                             its scratch; at least kpz_device_bytes(L) bytes,
                             256-byte aligned                                        */
    size_t dev_bytes;     /* size of dev_buf                                        */
    uint32_t decomposition; /* device layer: 0 = dead-border tiles with a random
                             origin (Sec. 3, the paper's KPZ scheme); 1 = the
                             double tiling the paper uses for KMC (Sec. 3.2):
                             the same tiles in four sets (tx & 1) + 2 (ty & 1),
                             swept one set at a time in an order drawn per sweep
                             from Philox (tag 5), no dead border. 1 needs
                             128 x 128 tiles and L >= 256. The work-group layer
                             (single-hit double tiling) is the same in both.
                             2 = no decomposition: the random-sequential
                             reference by colour classes (4 * 2^m sub-steps per
                             sweep, each attempting a random 2^-m subset of one
                             period-2 sublattice, m = colour_sparsity);
                             3 = dead borders at both layers (the paper's
                             earlier KPZ scheme, Sec. 3.1): the dead-border
                             tiles of 0, and inside each tile 16 rounds of
                             4 x 4 blocks anchored at a random offset, each
                             attempting one random site of its 3 x 3 interior
                             (Philox tags 9-11); 4 = no decomposition:
                             random-sequential updates equal bit for bit to
                             making the L^2 attempts of a sweep one at a time
                             (attempt a at the site drawn from Philox tag 4),
                             run as rounds of non-neighbouring sites whose
                             next attempt is the earliest around them; needs
                             L <= 8192, allocates about 20 L^2 bytes of
                             scratch itself (not in kpz_device_bytes) and
                             synchronises the stream every sweep.
                             2, 3 and 4 need 128 x 128 tiles                   */
    uint32_t cell;        /* work-group layer cell edge (Sec. 3.1): 4 (0 = 4):
                             4 x 4 cells, 2 x 2 quadrant sets, 16 rounds per
                             sweep; or 2: the C = 2 limit, 2 x 2 cells whose
                             1 x 1 quadrants are the sets, 4 rounds per sweep,
                             no position draw (needs 128 x 128 tiles and
                             decomposition 0)                                  */
    uint32_t colour_sparsity; /* decomposition 2: m in 1..4 (0 = 3); the bias
                             against one attempt at a time is of order 2^-m   */
} kpz_opts;

/* Roughness at the current time (eq. Wdef). Heights are taken in the gauge
 * h(0,0) = 0 (relative heights); W^2 does not depend on the gauge.
 * S2 = sum_h2_hi * 2^64 + sum_h2_lo, exact.                                  */
typedef struct {
    uint64_t t_mcs;       /* sweeps done since kpz_init                          */
    uint64_t n_sites;     /* L*L                                                 */
    int64_t sum_h;        /* S1 = sum of relative heights                        */
    uint64_t sum_h2_lo;   /* S2 = sum of squared relative heights, low 64 bits   */
    uint64_t sum_h2_hi;   /*   high 64 bits                                      */
    int64_t h00;          /* absolute height of site (0,0) (0 at the flat start) */
    double w2;            /* (N*S2 - S1^2) / N^2, numerator exact in 128 bits    */
} kpz_rough;

/* Device bytes a context of lateral size L needs (lattice + scratch), or 0 if
 * L is not a valid size. */
size_t kpz_device_bytes(uint32_t L);

/* Create a lattice and set it to the flat start (Sec. 2.1): heights
 * h(i,j) = (i+j) & 1, so W^2 = 1/4. `init` must be 0 (flat start).
 * Preconditions (KPZ_EINVAL otherwise, checked before any allocation):
 *   L a power of two with 128 <= L <= 262144 (2^18: 8 GiB of lattice at one
 *   bit per site, kpz_device_bytes(L) in all); 0 <= p, q <= 1 (no NaN);
 *   bx = 128 (or 0), by = 128 or 256 (or 0). p and q are quantised to multiples of 2^-16
 *   (T = min(65536, floor(x*65536 + 0.5))): attempts accept with U < T for a
 *   uniform 16-bit U. `sample` is the realisation index that enters the
 *   Philox counter next to the seed.                                          */
kpz_status kpz_init(kpz_ctx** out, uint32_t L, double p, double q, uint64_t seed,
                    uint32_t sample, int init, const kpz_opts* opts);

/* Return the lattice to the flat start (Sec. 2.1) with t = 0 and h(0,0) = 0,
 * keeping L, p, q, seed, sample and the device memory. Queued on the stream. */
kpz_status kpz_reset(kpz_ctx* ctx);

/* Queue n_mcs sweeps (n_mcs * L*L attempts) on the context's stream and
 * return; errors of the queued work surface at the next synchronising call. */
kpz_status kpz_run(kpz_ctx* ctx, uint64_t n_mcs);

/* Exact height sums and W^2 at the current time (eq. Wdef, Sec. 2.1).
 * Synchronises the stream. */
kpz_status kpz_roughness(kpz_ctx* ctx, kpz_rough* out);

/* Heights of all sites into host_out[j*L + i] (caller owns L*L int64).
 * absolute = 0: gauge h(0,0) = 0; absolute != 0: the absolute heights, i.e.
 * the relative ones plus the tracked height of site (0,0). Synchronises.     */
kpz_status kpz_heights(kpz_ctx* ctx, int64_t* host_out, int absolute);

/* Slopes in the packed exchange format into host_out (caller owns L*L/16
 * uint32). Synchronises. */
kpz_status kpz_slopes(kpz_ctx* ctx, uint32_t* host_out);

/* Replace the lattice by host_in (packed exchange format, L*L/16 words, a
 * valid surface: every row of sigma_x and every column of sigma_y sums to
 * zero), set the absolute height of site (0,0) to h00 and the sweep counter
 * to t_mcs. Validity is the caller's responsibility. Synchronises.          */
kpz_status kpz_set_slopes(kpz_ctx* ctx, const uint32_t* host_in, int64_t h00, uint64_t t_mcs);

/* Checkpoints (not in the paper; they let a long run such as the L = 2^16
 * job stop and resume). kpz_ckpt_save writes the context's whole state to
 * the file `path` (created or truncated):
 *   header   "KPZCKPT1", version 1, L, p, q (as given to kpz_init), the
 *            thresholds Tp, Tq, seed, sample, tile shape (bx, by), the device-layer
 *            decomposition, cell edge and colour sparsity (kpz_opts), the sweep
 *            counter t_mcs and the absolute height of site (0,0);
 *   payload  the lattice in the packed exchange format (L*L/16 uint32,
 *            row-major, as kpz_slopes), written in bands;
 *   trailer  a 64-bit FNV-1a checksum over the header and payload taken as
 *            little-endian 64-bit words.
 * kpz_ckpt_load creates a new context (*out, owned by the caller) from such a
 * file; opts supplies the execution options (run, warps_per_cta, stream,
 * dev_buf) as in kpz_init, and its bx, by must be 0 or equal the file's tile
 * shape. Running the loaded context gives the same lattices, bit for bit, as
 * the uninterrupted run. Both synchronise. Errors: KPZ_ECKPT for file and
 * format problems (nothing is created on load), KPZ_EINVAL for null
 * arguments or conflicting opts, otherwise as kpz_init / kpz_slopes.        */
kpz_status kpz_ckpt_save(kpz_ctx* ctx, const char* path);
kpz_status kpz_ckpt_load(kpz_ctx** out, const char* path, const kpz_opts* opts);

/* Throughput probe of the integer logic pipe that bounds the sweep (not in
 * the paper): one wave of CTAs runs independent chains of three-input XORs
 * (LOP3) on the current device; *lane_ops_per_s receives the measured rate
 * in lane operations per second and *kernel_ms (may be NULL) the kernel's
 * time. Synchronises its own stream. KPZ_EINVAL for a null output,
 * KPZ_ECUDA if a CUDA call fails.                                            */
kpz_status kpz_alu_peak(double* lane_ops_per_s, double* kernel_ms);

/* Device pointer of the lattice and its size in bytes, L*L/8 (for callers that
 * keep the lattice resident and time kernels on the context stream). */
kpz_status kpz_device_lattice(kpz_ctx* ctx, void** dev_ptr, size_t* bytes);

/* ------------------------------------------------------------------------ */
/* Batched ensemble: many independent realisations in one persistent launch. */
/* ------------------------------------------------------------------------ */
/* Each realisation is its own lattice run exactly as kpz_init + kpz_run would
 * run it (flat start, Sec. 2.1; decomposition of Sec. 3; same Philox streams),
 * so its W^2 sums equal those of a kpz_ctx with the same arguments. The paper
 * runs one lattice per GPU (Sec. 4); this call serves ensembles of unequal
 * lattices, whose small members alone would leave most of the GPU idle.    */
typedef struct kpz_batch kpz_batch;

typedef struct {
    uint32_t L;          /* lateral size: power of two, 128 <= L <= 131072        */
    double p, q;         /* attachment / detachment probabilities (eq. rule)      */
    uint64_t seed;       /* Philox key                                            */
    uint32_t sample;     /* realisation index (Philox counter word)               */
    uint32_t n_mcs;      /* sweeps to run                                         */
} kpz_spec;

typedef struct {
    void* stream;          /* cudaStream_t (NULL = default stream)                 */
    uint32_t n_samples;    /* log-spaced W^2 times up to the longest run (0 = 64);
                              every realisation is also sampled at its own end    */
    int autotune;          /* != 0: time a short probe of the ensemble for every
                              (tiles per run, warps per block), then for fewer
                              resident blocks per SM, and keep the fastest (these
                              choices never change the results); with tile_y = 0
                              also choose the tile height                        */
    uint32_t run;          /* tiles per run when not tuning (power of two, 0 = 4)  */
    uint32_t warps_per_cta;/* 1..8 (0 = 8)                                         */
    uint32_t ctas_per_sm;  /* resident blocks per SM (0 = as many as fit)          */
    uint32_t timeout_ms;   /* bound of every device-side wait (0 = 10000)          */
    int32_t test_block;    /* tests only: index (in run-length order, longest
                              first) of a realisation whose waits can never
                              succeed, to exercise the timeout; -1 = none        */
    uint32_t tile_y;       /* tile height for every realisation: 128 or 256
                              (256 needs every L >= 256). 0: 128, or, with
                              autotune, the faster of the two on the probe. The
                              tile shape is part of the schedule (Sec. 3.1): a
                              member equals the single-lattice run with the same
                              tile shape (kpz_opts.by), bit for bit            */
} kpz_batch_opts;

typedef struct {
    uint32_t run, warps_per_cta, ctas_per_sm, grid;  /* chosen execution knobs       */
    int graph;                                       /* 1: launched from a CUDA graph */
    uint64_t items;                                  /* work items in the queue       */
    uint32_t n_probe;                                /* autotune probes timed         */
    double probe_ms[8];                              /* their times                   */
    uint32_t tile_y;                                 /* tile height used (128, 256)   */
} kpz_batch_info;

/* Validate the specs (KPZ_EINVAL: bad L, p or q), allocate all lattices and
 * tables (KPZ_ENOMEM), optionally autotune, and capture the run in a graph.
 * opts may be NULL (defaults; test_block then -1).                          */
kpz_status kpz_batch_create(kpz_batch** out, const kpz_spec* specs, uint32_t n,
                            const kpz_batch_opts* opts);
/* Run every realisation from the flat start to its n_mcs with W^2 sampled at
 * the batch's sample times: one persistent cooperative launch. Synchronises.
 * KPZ_ETIMEOUT if a device-side wait ran out of time (the launch then stops
 * early and the batch may be run again).                                    */
kpz_status kpz_batch_run(kpz_batch* b);
/* Sample times (ascending, starting at 0). *n: capacity in, count out; times
 * may be NULL to query the count.                                           */
kpz_status kpz_batch_times(const kpz_batch* b, uint64_t* times, uint32_t* n);
/* Exact sums after kpz_batch_run, caller order, row-major [spec][time]
 * (n x n_times each); entries for times beyond a spec's n_mcs are 0. h00
 * (may be NULL): absolute height of site (0,0) of each lattice at its end.  */
kpz_status kpz_batch_sums(const kpz_batch* b, int64_t* S1, uint64_t* S2_lo, uint64_t* S2_hi,
                          int64_t* h00);
/* W^2 = (N S2 - S1^2) / N^2 (eq. Wdef), n x n_times, NaN beyond a spec's end. */
kpz_status kpz_batch_w2(const kpz_batch* b, double* w2);
kpz_status kpz_batch_get_info(const kpz_batch* b, kpz_batch_info* out);
void kpz_batch_free(kpz_batch* b);

/* ------------------------------------------------------------------------ */
/* Learned surrogate of W^2(t; L, p, q) (not part of the paper).             */
/* ------------------------------------------------------------------------ */
/* A 4-128-128-128-1 multilayer perceptron with GELU hidden units, bfloat16
 * weights and float32 arithmetic, trained by the library's own forward,
 * backward and Adam kernels. Parameters: one float32 vector of 33793 values,
 * W1 (128 x 4, row-major), b1 (128), W2 (128 x 128), b2, W3 (128 x 128), b3,
 * w4 (128), b4 (1). Inputs: n rows of 4 float32 features; targets: n float32.
 * The loss is the mean squared error. Gradients are reduced in a fixed order:
 * a call with the same inputs gives the same result. The 128 x 128 layers run
 * on the tcgen05 tensor cores with waits bounded in time: predict, loss_grad
 * and train return KPZ_ETIMEOUT if one ran out (the results are then
 * invalid; the handle stays usable), KPZ_ECUDA on a CUDA error.            */
typedef struct kpz_mlp kpz_mlp;
/* Upload initial parameters (caller-chosen initialisation); stream may be NULL. */
kpz_status kpz_mlp_create(kpz_mlp** out, const float* params, void* stream);
/* Current float32 master parameters (33793 values).                         */
kpz_status kpz_mlp_params(kpz_mlp* m, float* params);
/* y[i] = network(x[i]) with the bfloat16 weights.                           */
kpz_status kpz_mlp_predict(kpz_mlp* m, const float* x, uint32_t n, float* y);
/* Mean squared error over the n samples and its gradient (33793 values).   */
kpz_status kpz_mlp_loss_grad(kpz_mlp* m, const float* x, const float* t, uint32_t n, float* loss,
                             float* grad);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr);
 * step s uses samples order[s*batch .. s*batch+batch-1] of (x, t), order
 * holding steps*batch indices < n. last_loss: the loss of the last minibatch
 * before its update. The Adam moments persist across calls.               */
kpz_status kpz_mlp_train(kpz_mlp* m, const float* x, const float* t, uint32_t n, const uint32_t* order,
                         uint32_t steps, uint32_t batch, float lr, float* last_loss);
void kpz_mlp_free(kpz_mlp* m);

/* Exact W^2 of a lattice the caller already holds on the device, without
 * allocating anything. The paper has no counterpart to this call; it exists
 * for callers that cannot call cudaMalloc when they need the width: processes
 * whose device memory is fully reserved by another framework's caching
 * allocator, or loops that must not allocate after start-up. It computes what
 * kpz_roughness computes.
 *   lattice_dev: the lattice in the engine's layout, as returned by
 *                kpz_device_lattice (L*L/8 bytes, read only), in the memory
 *                of the current device;
 *   L:           its lateral size, a power of two with 128 <= L <= 131072;
 *   parity:      the parity of the absolute height of site (0,0) of the
 *                surface the lattice started from (0 for the flat start, h00 & 1
 *                after kpz_set_slopes);
 *   stream:      cudaStream_t to queue on (NULL = default stream); the call
 *                synchronises it;
 *   out:         host struct; t_mcs and h00 are set to 0 (this call has no
 *                context that knows them).
 * Scratch: one static device array of 512 KiB + 256 B per GPU that loads the
 * library, held until the process exits. L above 131072 returns KPZ_ERANGE;
 * a null pointer or an L that is not a power of two >= 128 returns
 * KPZ_EINVAL. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the rest
 * of the process; make that first call before any stream capture, and do not
 * call this function again after a reset of that device (cudaDeviceReset),
 * which invalidates the kept address. All calls share the array, which keeps the last
 * call's contents; the call clears what must start at zero. Calls that
 * overlap on the GPU (other streams, other host threads) race on the array. */
kpz_status kpz_roughness_static(const void* lattice_dev, uint32_t L, uint32_t parity,
                                void* stream, kpz_rough* out);

/* Number of kernels this library has launched in the process so far (all
 * contexts); lets a caller count the GPU work inside a timed region. */
uint64_t kpz_launch_count(void);

void kpz_free(kpz_ctx* ctx);
const char* kpz_strerror(kpz_status st);
/* Last error message of the context (empty string if none). */
const char* kpz_last_error(const kpz_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* KPZ_H */
