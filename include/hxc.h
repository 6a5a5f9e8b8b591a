/*
 * hxc.h -- C ABI of the B300 heat-stencil library.
 *
 * The calls follow the paper's programming model (Sec. 3.1 "Futurization",
 * Sec. 4 "Design of the implementation"): a device owns asynchronous work
 * queues, a buffer is device memory with asynchronous copies to and from the
 * host, a kernel launch takes buffers as arguments, and every asynchronous
 * call returns a future that later calls take as dependencies and that host
 * code composes with then / when_all / wait_all.  The work carried by those
 * futures is the explicit (forward-time, centred-space) heat stencil in
 * 1D/2D/3D, a batched variable-diffusivity form and its discrete adjoint.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Status.  Every call returns hxc_status.  Argument errors are reported
 *    synchronously and create no future.  Errors of asynchronous work (a
 *    CUDA error, a failing host continuation) are stored in the future of
 *    that work; an operation whose dependency failed does not run and its
 *    future holds HXC_E_DEP_FAILED.  hxc_last_error() gives a thread-local
 *    description of the last synchronous error.
 *  - Handles (hxc_device, hxc_buffer, hxc_future, hxc_graph) are opaque and
 *    reference counted.  The caller releases each handle it receives exactly
 *    once.  A future keeps the buffers its operation uses alive until the
 *    future itself is released.
 *  - Host pointers given to asynchronous copies must stay valid and
 *    unmodified until the copy's future is ready (as for cudaMemcpyAsync).
 *    Page-locked memory from hxc_host_alloc overlaps with other work;
 *    pageable memory is accepted but the copy may be staged.
 *  - Stream slots.  A device has up to HXC_MAX_SLOTS asynchronous queues
 *    (CUDA streams, created on first use).  Work on one slot runs in issue
 *    order; work on different slots is ordered only by futures.
 *  - Threads.  All calls are thread-safe.  While a thread captures a graph
 *    on a device, work that other threads issue to that device waits until
 *    the capture ends (hxc_graph_begin).  Host continuations run on an
 *    internal worker pool, never on CUDA's callback thread.
 *  - Waits are bounded: hxc_future_wait takes a timeout, and no kernel of
 *    the library waits on another CTA or on the host.
 *
 * Data layouts
 *  - 1D fields: n contiguous doubles, periodic.
 *  - 2D fields: row-major ny x nx doubles, element (i, j) = (y, x) at
 *    i * nx + j, Dirichlet-zero ghost ring outside the field.
 *  - 3D fields: nz x ny x nx floats, x fastest, periodic.
 *  - Batches: problems packed back to back, problem p a row-major side_p x
 *    side_p block starting at element offset_p.
 */
#ifndef HXC_H
#define HXC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HXC_MAX_SLOTS 256
#define HXC_ABI_VERSION 1

typedef struct hxc_device_t *hxc_device;
typedef struct hxc_buffer_t *hxc_buffer;
typedef struct hxc_future_t *hxc_future;
typedef struct hxc_graph_t *hxc_graph;

typedef enum {
    HXC_OK = 0,
    HXC_E_INVALID = 1,      /* bad argument or handle                         */
    HXC_E_NOMEM = 2,        /* device or host allocation failed               */
    HXC_E_CUDA = 3,         /* CUDA runtime error (see hxc_last_error)         */
    HXC_E_TIMEOUT = 4,      /* a bounded wait ran out                         */
    HXC_E_DEP_FAILED = 5,   /* a dependency failed; this operation did not run */
    HXC_E_CALLBACK = 6,     /* a host continuation returned an error          */
    HXC_E_UNSUPPORTED = 7,  /* valid request this build does not support      */
    HXC_E_NODEV = 8         /* no CUDA device satisfies the request           */
} hxc_status;

/* Host continuation for hxc_future_then: runs on the worker pool once the
 * antecedent future is ready and succeeded.  Returning anything other than
 * HXC_OK stores HXC_E_CALLBACK in the continuation's future. */
typedef hxc_status (*hxc_host_fn)(void *user);

/* Launch configuration (Listing 2 exposes grid and block to the user,
 * Sec. 4.2).  Passing NULL lets the library choose (autotuned).  Every
 * built-in kernel is correct for any grid (grid-stride loops); the block
 * must be a multiple of 32 threads within the kernel's supported range. */
typedef struct {
    uint32_t grid[3];
    uint32_t block[3];
} hxc_launch_cfg;

/* ------------------------------------------------------------------ status */

const char *hxc_status_string(hxc_status s);
/* Thread-local text of the last synchronous error of this thread (never NULL). */
const char *hxc_last_error(void);
int hxc_abi_version(void);
/* Drains the worker pool and joins its threads.  Optional; call before
 * process exit when continuations may still be running. */
hxc_status hxc_shutdown(void);

/* ----------------------------------------------------------------- devices */

/* Sec. 4.1, Listing 1: all local CUDA devices whose compute capability is at
 * least (min_major, min_minor).  Writes up to `cap` new device handles to
 * `out` and the number of matching devices to *n_out.  Remote devices of the
 * paper's distributed setting are not supported (single node, single GPU).
 * Returns HXC_E_NODEV when no device matches. */
hxc_status hxc_get_all_devices(int min_major, int min_minor, hxc_device *out, int cap,
                               int *n_out);
/* Compute capability, SM count and global memory of a device. */
hxc_status hxc_device_info(hxc_device dev, int *major, int *minor, int *sm_count,
                           size_t *global_mem);
/* Blocks until every slot of the device is idle (cudaDeviceSynchronize
 * semantics restricted to this library's streams). */
hxc_status hxc_device_synchronize(hxc_device dev);
/* The CUDA stream (cudaStream_t) behind a slot, created if needed. */
hxc_status hxc_device_stream(hxc_device dev, int slot, void **stream);
hxc_status hxc_device_retain(hxc_device dev);
hxc_status hxc_device_release(hxc_device dev);

/* ----------------------------------------------------------- host memory */

/* Page-locked host allocation (Listing 2 allocates its host data with
 * cudaMallocHost).  Free with hxc_host_free. */
hxc_status hxc_host_alloc(size_t bytes, void **p);
hxc_status hxc_host_free(void *p);

/* ----------------------------------------------------------------- buffers */

/* Sec. 4, "buffer": `bytes` of device memory on `dev` (cudaMalloc, Listing 2
 * line "create_buffer").  Contents are undefined until written. */
hxc_status hxc_device_create_buffer(hxc_device dev, size_t bytes, hxc_buffer *out);
/* Wraps existing device memory (for example a torch tensor) without taking
 * ownership: the memory must outlive the buffer and every future using it. */
hxc_status hxc_buffer_wrap(hxc_device dev, void *device_ptr, size_t bytes, hxc_buffer *out);
hxc_status hxc_buffer_device_ptr(hxc_buffer buf, void **device_ptr, size_t *bytes);
hxc_status hxc_buffer_retain(hxc_buffer buf);
hxc_status hxc_buffer_release(hxc_buffer buf);

/* Asynchronous host->device copy of `bytes` from `host` into the buffer at
 * byte offset `off` (Listing 2 "enqueue_write", cudaMemcpyAsync).  Runs on
 * stream slot `slot` after every future in deps[0..ndeps) is ready. */
hxc_status hxc_buffer_enqueue_write(hxc_buffer buf, size_t off, size_t bytes, const void *host,
                                    int slot, const hxc_future *deps, int ndeps,
                                    hxc_future *out);
/* Asynchronous device->host copy (Listing 2 "enqueue_read"). */
hxc_status hxc_buffer_enqueue_read(hxc_buffer buf, size_t off, size_t bytes, void *host,
                                   int slot, const hxc_future *deps, int ndeps,
                                   hxc_future *out);
/* Synchronous read (Listing 2 "enqueue_read_sync"): enqueue, then wait
 * without a time limit. */
hxc_status hxc_buffer_enqueue_read_sync(hxc_buffer buf, size_t off, size_t bytes, void *host,
                                        int slot, const hxc_future *deps, int ndeps);
/* Asynchronous device->device copy between buffers of the same device. */
hxc_status hxc_buffer_enqueue_copy(hxc_buffer dst, size_t dst_off, hxc_buffer src,
                                   size_t src_off, size_t bytes, int slot,
                                   const hxc_future *deps, int ndeps, hxc_future *out);
/* Asynchronous strided 2D copies: `rows` rows of `row_bytes` bytes; the
 * buffer side starts at byte offset `off` with pitch `buf_pitch`, the host
 * side at `host` with pitch `host_pitch` (cudaMemcpy2DAsync). */
hxc_status hxc_buffer_enqueue_write_2d(hxc_buffer buf, size_t off, size_t buf_pitch,
                                       const void *host, size_t host_pitch, size_t row_bytes,
                                       size_t rows, int slot, const hxc_future *deps,
                                       int ndeps, hxc_future *out);
hxc_status hxc_buffer_enqueue_read_2d(hxc_buffer buf, size_t off, size_t buf_pitch,
                                      void *host, size_t host_pitch, size_t row_bytes,
                                      size_t rows, int slot, const hxc_future *deps,
                                      int ndeps, hxc_future *out);

/* ----------------------------------------------------------------- futures */

/* Sec. 3.1: futures compose with then and when_all; wait_all is a barrier.
 * A future is ready when its operation finished; its status is then final. */
hxc_status hxc_future_is_ready(hxc_future f, int *ready);
/* Waits up to timeout_ns nanoseconds (< 0: no limit).  Returns the future's
 * final status, or HXC_E_TIMEOUT if it did not become ready in time (the
 * future stays valid and may be waited on again). */
hxc_status hxc_future_wait(hxc_future f, int64_t timeout_ns);
/* Waits for every future (Listing 2 "wait_all"); returns the first
 * non-OK status in array order, HXC_E_TIMEOUT if the time ran out. */
hxc_status hxc_wait_all(const hxc_future *fs, int n, int64_t timeout_ns);
/* Attaches a host continuation (Sec. 3.1 "then").  `out` becomes ready with
 * fn's status after fn returned; fn does not run if f failed. */
hxc_status hxc_future_then(hxc_future f, hxc_host_fn fn, void *user, hxc_future *out);
/* Joins futures (Sec. 3.1 "when_all").  When every input is device work the
 * join is done on the device (no host round trip). */
hxc_status hxc_when_all(const hxc_future *fs, int n, hxc_future *out);
/* An already-ready future holding `status`. */
hxc_status hxc_make_ready_future(hxc_status status, hxc_future *out);
/* A future completed later by hxc_promise_set (host-side producer). */
hxc_status hxc_promise_create(hxc_future *out);
hxc_status hxc_promise_set(hxc_future promise, hxc_status status);

/* Host-side fault injection for testing failure handling (the paper's
 * futures carry errors, Sec. 3.1; it has no injection facility): after
 * `after_ops` further device operations (copies, kernel launches, joins;
 * 0 = the next one), one operation is not enqueued and its future completes
 * with `status` (not HXC_OK), exactly as if its CUDA call had returned an
 * error; operations that depend on it complete with HXC_E_DEP_FAILED and
 * their continuations do not run.  Nothing faults on the device and the
 * device stays usable.  Inside a graph capture the capture fails.  Process-
 * wide and one-shot; after_ops < 0 disarms.  Returns HXC_E_INVALID for
 * status == HXC_OK with after_ops >= 0. */
hxc_status hxc_debug_inject(int64_t after_ops, hxc_status status);
/* The paper has no counterpart to this call.  Device-side waits of the
 * library's kernels are bounded (the 3D form 7 waits on shared-memory
 * barriers for its TMA copies); a wait that runs out sets a bit in a
 * device-wide record and its CTA leaves without finishing its work.  This
 * call synchronises the device's slots, then reads and clears the record:
 * *flags = 0 when no wait ran out since the last call, bit 0 set when a 3D
 * TMA wait did. */
hxc_status hxc_debug_wait_errors(hxc_device dev, uint32_t *flags);
/* Interop with foreign CUDA streams (e.g. torch's current stream):
 * a future for everything issued so far on `stream` ... */
hxc_status hxc_future_from_stream(hxc_device dev, void *stream, hxc_future *out);
/* ... and making `stream` wait for a future (device-side, no host wait). */
hxc_status hxc_future_stream_wait(hxc_future f, void *stream);
hxc_status hxc_future_retain(hxc_future f);
hxc_status hxc_future_release(hxc_future f);

/* --------------------------------------------------------- kernel launches */

/* Built-in kernels (the paper's "program.run(args, name, grid, block)",
 * Sec. 4.2, with a fixed kernel table instead of run-time compilation). */
typedef enum {
    /* Listing 2: result[0] = sum of n uint32 values (64-bit result). */
    HXC_K_SUM_U32 = 1,
    /* Sec. 5.1.1: out_i = 0.5 in_{i-1} + in_i + 0.5 in_{i+1}, periodic. */
    HXC_K_PRK_STENCIL = 2,
    /* 1D FTCS: dst[lo, lo+count) = `steps` periodic steps of src.  steps > 1
     * reads a halo of width `steps` from src (temporal blocking).  Every
     * point rounds t = fma(-2, u, ul + ur), u' = fma(r, t, u) in FP64. */
    HXC_K_HEAT1D = 3,
    /* 2D FTCS step on the tile [y0, y0+ty) x [x0, x0+tx), zero outside the
     * field; every point rounds t = fma(-4, u, (uN + uW) + (uE + uS)),
     * u' = fma(r, t, u) in FP64, so any tiling gives the same bits. */
    HXC_K_HEAT2D = 4,
    /* Tile snapshot and squared norm: copies the tile of src into the compact
     * ty x tx buffer snap (optional) and stores sum(u^2) of the tile in
     * sums[sum_index] with a fixed reduction order. */
    HXC_K_TILE_NORM2 = 5,
    /* 3D FTCS, FP32, periodic, `steps` (1..4) fused steps per launch; every
     * cell rounds t = fma(-6, u, (((x- + x+) + (y- + y+)) + z-) + z+),
     * u' = fma(r, t, u) in FP32, so any blocking gives the same bits. */
    HXC_K_HEAT3D = 6,
    /* Variable-diffusivity FTCS step (flux form, arithmetic face mean). */
    HXC_K_VARCOEF2D = 7,
    /* Adjoint step with kappa-gradient accumulation. */
    HXC_K_ADJOINT2D = 8,
    /* Sec. 5.1.2 partition kernel k, in place on x[offset, offset+n):
     * x_i <- sqrt(sin(x_i)^2 + cos(x_i)^2), 1 up to rounding. */
    HXC_K_PARTITION = 9,
    /* Sec. 5.1.3 Mandelbrot image (escape time, binary32). */
    HXC_K_MANDELBROT = 10
} hxc_kernel_id;

typedef struct { hxc_buffer input, result; int64_t n; } hxc_sum_args;
typedef struct { hxc_buffer in, out; int64_t n; } hxc_prk_args;
typedef struct {
    hxc_buffer src, dst;
    int64_t n, lo, count;  /* field length, first updated point, points updated */
    double r;              /* diffusion number dt/h^2 (stable for r <= 1/2) */
    int32_t steps;         /* >= 1 */
} hxc_heat1d_args;
typedef struct {
    hxc_buffer src, dst;
    int64_t ny, nx;        /* field shape */
    int64_t y0, x0, ty, tx; /* updated tile */
    double r;              /* stable for r <= 1/4 */
} hxc_heat2d_args;
typedef struct {
    hxc_buffer src, snap, sums; /* snap may be NULL */
    int64_t ny, nx, y0, x0, ty, tx;
    int64_t sum_index;     /* element of sums (doubles) receiving sum(u^2) */
} hxc_tile_norm2_args;
typedef struct {
    hxc_buffer src, dst;
    int64_t nz, ny, nx;
    float r;               /* stable for r <= 1/6 */
    int32_t steps;         /* 1..4 */
} hxc_heat3d_args;
typedef struct {
    hxc_buffer src, dst, kappa;
    int64_t ny, nx;
    double c;              /* dt/h^2; stable for c * sum_f k_f <= 1 */
} hxc_varcoef2d_args;
typedef struct {
    hxc_buffer lam_in, lam_out, u, kappa, grad_kappa;
    int64_t ny, nx;
    double c;
} hxc_adjoint2d_args;
typedef struct { hxc_buffer x; int64_t n, offset; } hxc_partition_args;
/* Sec. 5.1.3.  Pixel (i, j), 0 <= i < width, 0 <= j < height, is the point
 * c = (x0 + i*dx) + (y0 + j*dy) i (each product and sum rounded to float).
 * Its escape count k is the first k < max_iter with |z_k|^2 > 4, where
 * z_0 = 0 and z_{k+1} = z_k^2 + c, else max_iter (a member).  One iteration
 * in binary32: xx = x*x, yy = y*y, test xx + yy > 4, Im z' = fma(x + x, y,
 * Im c), Re z' = (xx - yy) + Re c.  rgb: width*height*3 bytes, row-major
 * RGB8; members black, else (9k, 5k, 13k) mod 256.  counts (may be NULL):
 * width*height int32.  width, height <= 2^24; max_iter >= 1; a launch
 * configuration, if given, has at most 256 threads per block. */
typedef struct {
    hxc_buffer rgb, counts;
    int64_t width, height;
    float x0, y0, dx, dy;
    int32_t max_iter, reserved;
} hxc_mandelbrot_args;

/* Launches kernel `id` with the argument struct `args` (of size args_size,
 * which must equal the struct's size) on stream slot `slot` after deps. */
hxc_status hxc_launch(hxc_device dev, hxc_kernel_id id, const void *args, size_t args_size,
                      const hxc_launch_cfg *cfg, int slot, const hxc_future *deps, int ndeps,
                      hxc_future *out);

/* ----------------------------------------- partition benchmark (Alg. 1) */

/* Sec. 5.1.2, Algorithm 1: the n doubles at host_x are split into `parts`
 * contiguous partitions (partition i holds [i*n/parts, (i+1)*n/parts)) and
 * issued as three loops over the partitions: partition i is written into
 * `work` (at least 8n bytes, same offsets) on stream slot i, the partition
 * kernel (HXC_K_PARTITION) runs on it after its write, and it is read back
 * into host_r after its kernel -- each operation a future of the public
 * calls.  host_r may equal host_x; both should be page-locked
 * (hxc_host_alloc) for the copies to overlap with the kernels.  The first
 * writes wait for deps.  *out completes when every partition is on the host
 * (with deps alone when n = 0).  1 <= parts <= 64. */
hxc_status hxc_partition_run(hxc_device dev, const double *host_x, double *host_r, int64_t n,
                             int parts, hxc_buffer work, const hxc_future *deps, int ndeps,
                             hxc_future *out);
/* The same three loops as plain CUDA runtime calls (cudaMemcpyAsync, kernel,
 * cudaMemcpyAsync) on the same stream slots, without futures, then a
 * synchronisation of each stream: the native comparison of Sec. 5.1.2.
 * Returns when the results are on the host. */
hxc_status hxc_partition_run_native(hxc_device dev, const double *host_x, double *host_r,
                                    int64_t n, int parts, hxc_buffer work);

/* ------------------------------------------- Mandelbrot images (Sec. 5.1.3) */

/* Writes an RGB8 image (height rows of width*3 bytes) as a PNG file: 8-bit
 * truecolour, no interlace, filter type 0 on every row, zlib level `level`
 * (-1 = zlib's default, 0..9).  Synchronous; HXC_E_INVALID on a bad
 * argument or an I/O error (hxc_last_error names the file). */
hxc_status hxc_png_write(const uint8_t *rgb, int64_t width, int64_t height, int level,
                         const char *path);

/* Sec. 5.1.3: one Mandelbrot image (HXC_K_MANDELBROT with *args, after
 * deps, on stream slot `slot`), read into host_rgb (width*height*3 bytes,
 * page-locked for an asynchronous copy), then written to `path` as by
 * hxc_png_write.  With async_write != 0 the call returns after issuing the
 * kernel and the copy; the file is written by a continuation on the worker
 * pool and *out completes when the file is closed, so the caller may issue
 * the next image (in other buffers) meanwhile -- the paper's asynchronous
 * write.  host_rgb must stay valid and unchanged until then.  With
 * async_write = 0 the call waits for the image, writes the file and returns
 * with *out ready (the paper's synchronous write). */
hxc_status hxc_mandelbrot_png(hxc_device dev, const hxc_mandelbrot_args *args, uint8_t *host_rgb,
                              const char *path, int level, int async_write, int slot,
                              const hxc_future *deps, int ndeps, hxc_future *out);

/* ---------------------------------------------------- run-time programs */

/* Sec. 4 "program" and Listing 2: user CUDA source compiled at run time
 * (NVRTC) for the device's architecture.  Creation reads the source
 * synchronously; hxc_program_build returns a future (Listing 2 adds it to
 * the futures it waits for); hxc_program_run launches a kernel of the
 * program with buffers (and values) as arguments and an explicit grid and
 * block (Listing 2, "run(args, name, grid, block)"), returning a future.
 * Every run of a program depends on the program's last build. */
typedef struct hxc_program_t *hxc_program;

/* A kernel argument: a buffer (passed as its device pointer) or, when buf is
 * NULL, `size` bytes at `value` (copied when hxc_program_run is called). */
typedef struct {
    hxc_buffer buf;
    const void *value;
    size_t size;
} hxc_kernel_arg;

hxc_status hxc_program_create_with_source(hxc_device dev, const char *source, const char *name,
                                          hxc_program *out);
/* Listing 2 "create_program_with_file". */
hxc_status hxc_program_create_with_file(hxc_device dev, const char *path, hxc_program *out);
/* Compiles the program and loads the kernels named in the comma-separated
 * list kernel_names (name expressions: plain names for extern "C" kernels,
 * C++ names otherwise).  `options` (may be NULL) are extra NVRTC options
 * separated by spaces.  The future holds HXC_E_INVALID on a compile error
 * (see hxc_program_build_log), HXC_E_UNSUPPORTED if NVRTC is unavailable. */
hxc_status hxc_program_build(hxc_program prog, const char *kernel_names, const char *options,
                             const hxc_future *deps, int ndeps, hxc_future *out);
/* Compiler output of the last build: copies up to cap-1 bytes and a NUL;
 * *len receives the full length. */
hxc_status hxc_program_build_log(hxc_program prog, char *buf, size_t cap, size_t *len);
hxc_status hxc_program_run(hxc_program prog, const char *kernel_name, const hxc_kernel_arg *args,
                           int nargs, const hxc_launch_cfg *cfg, int slot, const hxc_future *deps,
                           int ndeps, hxc_future *out);
hxc_status hxc_program_release(hxc_program prog);

/* ------------------------------------------------------------------ graphs */

/* Captures every operation subsequently issued to `dev` by this thread into
 * a CUDA graph.  Futures created during capture may be used as dependencies
 * inside the capture only.  Dependencies from before the capture must be
 * ready.  Host continuations cannot be captured (HXC_E_UNSUPPORTED).
 * Operations that other threads (or the worker pool) issue to `dev` during
 * the capture wait until it ends, as does another thread's hxc_graph_begin;
 * a wait that exceeds 60 s gives HXC_E_TIMEOUT.  So the capturing thread must
 * not wait for another thread's operation on the same device before it ends
 * the capture. */
hxc_status hxc_graph_begin(hxc_device dev);
hxc_status hxc_graph_end(hxc_device dev, hxc_graph *out);
/* Replays the graph on slot `slot` after deps. */
hxc_status hxc_graph_launch(hxc_graph g, int slot, const hxc_future *deps, int ndeps,
                            hxc_future *out);
hxc_status hxc_graph_node_count(hxc_graph g, size_t *nodes);
hxc_status hxc_graph_release(hxc_graph g);

/* ------------------------------------------------- whole-run entry points */

typedef enum {
    /* one launch per partition and step, ordered by futures (baseline) */
    HXC_MODE_PLAIN = 0,
    /* the same operations captured once into a CUDA graph and replayed */
    HXC_MODE_GRAPH = 1,
    /* fewest launches: temporal blocking / whole-domain / persistent kernels */
    HXC_MODE_FUSED = 2
} hxc_mode;

/* Counters filled by the run entry points (optional). */
typedef struct {
    int64_t kernel_launches;   /* kernels launched by the host (graph replays count their nodes) */
    int64_t graph_launches;
    int64_t copies;
    int64_t host_tasks;        /* host continuations run */
    int64_t h2d_bytes, d2h_bytes;
} hxc_run_stats;

/* 1D periodic FTCS over n points in `parts` equal partitions: `steps` steps
 * with diffusion number r.  u holds the initial field and receives the
 * result; tmp is scratch of the same size.  Each partition reads a halo from
 * its neighbours: in PLAIN and GRAPH mode step s of partition p runs after
 * step s-1 of p-1, p and p+1; FUSED mode advances `steps_per_launch` steps
 * per launch (0: the tuned count, knob heat1d.steps_per_launch, whose
 * default 0 puts all steps in one launch).  The steps' arithmetic is given
 * under hxc_heat1d_step_kinds.  Results are bit-identical for every
 * partition count, mode and steps per launch. */
hxc_status hxc_heat1d_run(hxc_device dev, hxc_buffer u, hxc_buffer tmp, int64_t n, int parts,
                          double r, int steps, hxc_mode mode, int steps_per_launch,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_run_stats *stats);

/* Step kinds of a 1D run (hxc_heat1d_run), as for the 2D runs
 * (hxc_heat2d_step_kinds) with s = ul + ur: counts[1] scaled steps,
 * v' = fma((1-2r)/r, v, s), 2 FP64 operations per point; counts[2] closing
 * steps, u' = fma(r^(m+1), s, ((1-2r) r^m) v), 3 operations; counts[0]
 * canonical steps, t = fma(-2, u, s), u' = fma(r, t, u), 3 operations (every
 * step when r is outside (0, 1/2] or r^-1 > 2^96).  The intervals are of
 * min(steps, 128) steps (what one captured graph holds), cut into groups of
 * at most M + 1 steps, M the largest m with r^-m <= 2^96 (48 at r = 1/4).
 * counts: 3 int64 written.  Host only, no device needed. */
hxc_status hxc_heat1d_step_kinds(double r, int steps, int64_t *counts);

typedef struct {
    int64_t ny, nx;            /* field shape */
    int64_t tiles_y, tiles_x;  /* partition grid; tiles may be ragged */
    double r;
    int32_t steps;
    int32_t snapshot_every;    /* 0: no snapshots */
    hxc_mode mode;
    /* Outputs, row-major [n_snapshots][tiles_y * tiles_x] (may be NULL):
     * host_norms: sqrt(sum u^2) per tile computed on the host from a
     *   device->host snapshot, as then-continuations overlapping the steps;
     * gpu_norms: the same norms reduced on the device. */
    double *host_norms;
    double *gpu_norms;
} hxc_heat2d_cfg;

/* 2D Dirichlet FTCS on device buffers: u (initial field, receives the
 * result) and tmp (scratch), each ny * nx doubles.  Snapshots are taken
 * after steps k * snapshot_every (k = 1, 2, ...).  *out becomes ready when
 * everything, host norms included, is done; *field_ready (optional) as soon
 * as u holds the result, possibly before the host norms finish.  The cfg
 * struct is copied; the norm arrays must stay valid until *out is ready.
 * When a dependency is unfinished host work the whole run is issued later
 * by the worker pool (stats then count nothing).  2D runs on one device are
 * issued one at a time (they share the device's snapshot rings and norm
 * rows): a run called while another thread issues one is queued and issued
 * by that thread right after, without blocking the caller (stats again
 * count nothing; errors then reach *out instead of the return value).
 * The steps' arithmetic is given under hxc_heat2d_step_kinds; it depends
 * on the step's index only, so results are bit-identical for every tile
 * grid and mode. */
hxc_status hxc_heat2d_run(hxc_device dev, hxc_buffer u, hxc_buffer tmp, const hxc_heat2d_cfg *cfg,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_future *field_ready, hxc_run_stats *stats);
/* The same run with a host-resident field: host_u0 is copied in tile by
 * tile, the result is copied out tile by tile into host_uT (may alias
 * host_u0).  Synchronous: returns when host_uT and the norms are written. */
hxc_status hxc_heat2d_run_host(hxc_device dev, const double *host_u0, double *host_uT,
                               const hxc_heat2d_cfg *cfg, hxc_run_stats *stats);
/* The asynchronous form: the uploads start after `deps`; *out completes
 * when host_uT holds the result and the run (its norms included) is done.
 * The library keeps two device field pairs per device for these calls and
 * gives them out in turn, so the uploads and downloads of one call overlap
 * the steps of the call issued before it; a call's uploads wait (on the
 * device) for the downloads of the call issued two before it, the last user
 * of its pair.  host_u0 must stay valid and host_uT untouched until *out is
 * ready; both should be page-locked (hxc_host_alloc) for the copies to
 * overlap.  Calls whose snapshot norms go to the same arrays must not
 * overlap (each run writes every entry).  The two field pairs grow to the
 * largest field used; a pair outgrown by a larger call stays allocated (an
 * operation still to be issued may hold it) until the process ends.
 * A call's steps also start after the device-norm copy of the 2D run
 * issued before it (measured: back-to-back calls 6% faster).  A call that
 * has to wait for unfinished host work (a dependency that is a promise or a
 * host continuation, or the call that used its field pair last) is issued
 * as a whole by the worker pool once every dependency is done; its stats
 * then count nothing.
 * Argument errors are returned synchronously with no future created; a
 * failure of a copy or of the run is stored in *out and does not affect
 * later calls. */
hxc_status hxc_heat2d_run_host_async(hxc_device dev, const double *host_u0, double *host_uT,
                                     const hxc_heat2d_cfg *cfg, const hxc_future *deps,
                                     int ndeps, hxc_future *out, hxc_run_stats *stats);

/* Step kinds of a 2D run (hxc_heat2d_run and its host forms; the streamed
 * run of the same steps without snapshots).  FTCS is linear,
 * u_{n+1} = r ((1 - 4r)/r u_n + s(u_n)) with s the four neighbours' sum, so
 * the runs carry the field scaled by r^-m after m steps and advance it with
 * one FMA after the sum: counts[1] "scaled" steps, v' = fma((1-4r)/r, v, s),
 * 3 FP64 operations per point; counts[2] "closing" steps back to true
 * values, u' = fma(r^(m+1), s, ((1-4r) r^m) v), 4 operations; counts[0]
 * canonical steps, t = fma(-4, u, s), u' = fma(r, t, u), 4 operations (every
 * step when r is outside (0, 1/4] or r^-1 > 2^96).  s is always
 * (uN + uW) + (uE + uS).  The steps are issued in intervals (snapshot_every
 * when snapshot norms are requested, else min(steps, 100)); each interval is
 * cut into groups of at most M + 1 steps, M the largest m with r^-m <= 2^96
 * (41 at r = 0.2), whose last step closes, so the field holds true values at
 * every snapshot and at the end.  The scaled field grows by at most 1/r per
 * step: inputs with |u| <= 2^927 stay finite.  counts: 3 int64 written.
 * Host only, no device needed. */
hxc_status hxc_heat2d_step_kinds(const hxc_heat2d_cfg *cfg, int64_t *counts);

/* 3D periodic FTCS in FP32 on an nz x ny x nx field (x fastest): u holds
 * the initial field and receives the result, tmp is scratch of the same
 * size.  PLAIN launches one step at a time, FUSED advances
 * `steps_per_launch` (1..4; 0: the tuned count, knob heat3d.steps_per_launch,
 * default 4) steps per launch with temporal blocking,
 * GRAPH captures the fused launches once and replays them.  All modes give
 * bit-identical results. */
/* The host half of the norms (a then-continuation of every snapshot in
 * hxc_heat2d_run) as a call of its own: out[i] = sqrt(sum of squares) of
 * the counts[i] doubles at arrays[i], one task per array on the worker
 * pool, in the same summation order as the run's continuations (blocks of
 * 64 squares over 8 accumulators, block sums pairwise).  Synchronous. */
hxc_status hxc_host_norms(const double *const *arrays, const int64_t *counts, int n, double *out);

/* The 2D run with the field in host memory and every step streamed through
 * the device (Algorithm 1 per step; the contrast Sec. 5.1.1 measures):
 * each of the tiles_y x tiles_x tiles (split as in hxc_heat2d_run) is copied
 * in with its one-cell halo, advanced one step and copied back, every step.
 * host_a holds the initial ny x nx field; host_b is the second host array
 * (the arrays alternate: after `steps` steps the result is in host_a if
 * steps is even, in host_b if odd; both are overwritten).  Both should be
 * page-locked (hxc_host_alloc) for copies to overlap.  sequential = 0:
 * every tile-step is a future on the tile's stream slot, after the
 * tile-steps of the previous step whose results its halo reads, so copies
 * and kernels of different tiles overlap; *out completes when the last
 * tile is back.  sequential != 0: the native sequential loop (copy in,
 * kernel, copy out, wait, tile after tile) on one stream; returns when done
 * with *out ready.  Results are bit-identical to hxc_heat2d_run. */
hxc_status hxc_heat2d_stream_run(hxc_device dev, double *host_a, double *host_b, int64_t ny,
                                 int64_t nx, int64_t tiles_y, int64_t tiles_x, double r, int steps,
                                 int sequential, const hxc_future *deps, int ndeps,
                                 hxc_future *out, hxc_run_stats *stats);

hxc_status hxc_heat3d_run(hxc_device dev, hxc_buffer u, hxc_buffer tmp, int64_t nz, int64_t ny,
                          int64_t nx, float r, int steps, hxc_mode mode, int steps_per_launch,
                          const hxc_future *deps, int ndeps, hxc_future *out,
                          hxc_run_stats *stats);

/* A batch of independent variable-diffusivity problems (Dirichlet-zero,
 * flux form with arithmetic face mean), `nprob` square problems of side
 * sides[p] packed back to back in u and kappa (problem p starts at element
 * sum_{q<p} sides[q]^2), each with its own c[p] = dt/h^2.  u holds the initial
 * fields and receives the results after `steps` steps.  sides and c are host
 * arrays read during the call.  PLAIN launches one kernel per problem and
 * step (plus one coefficient kernel per problem), GRAPH replays a captured
 * sequence of batched per-step launches, FUSED runs one persistent launch in
 * which every CTA takes whole problems (largest first) from a queue.  All
 * modes give bit-identical results.  Uses device scratch (a second field,
 * three coefficient arrays, the problem list and a work counter) shared by
 * all batch runs on the device: a run must depend on the future of any
 * earlier batch run it could otherwise overlap with. */
hxc_status hxc_varcoef_batch_run(hxc_device dev, hxc_buffer u, hxc_buffer kappa,
                                 const int64_t *sides, const double *c, int64_t nprob, int steps,
                                 hxc_mode mode, const hxc_future *deps, int ndeps,
                                 hxc_future *out, hxc_run_stats *stats);

/* Squared error and adjoint seed: loss[0] = sum_i (u_i - t_i)^2 (fixed
 * reduction order) and, if lam is not NULL, lam_i = 2 (u_i - t_i).  u, t and
 * lam hold n doubles, loss one double. */
hxc_status hxc_sqerr_seed(hxc_device dev, hxc_buffer u, hxc_buffer t, hxc_buffer lam,
                          hxc_buffer loss, int64_t n, int slot, const hxc_future *deps,
                          int ndeps, hxc_future *out);

/* Reverse-mode gradient of a scalar loss of u^T through `steps`
 * variable-diffusivity steps on one ny x nx problem: given u0, kappa and
 * lamT = dL/du^T, computes gk = dL/dkappa and gu0 = dL/du0 (= lambda^0),
 * and the final state into uT if uT is not NULL.  The forward states are
 * kept only every `every` steps (0: every = ceil(sqrt(steps))) and each
 * segment is recomputed from its checkpoint before its adjoint steps;
 * every = 1 stores every state.  c is fixed (not differentiated).  FUSED
 * fuses the adjoint step with the kappa-gradient accumulation, PLAIN
 * launches them separately, GRAPH replays the captured fused sequence.  The
 * results are bit-identical for every mode and every `every`.  Device
 * scratch (coefficients, checkpoints, the segment store, work and adjoint
 * fields) is shared by the adjoint runs of a device: order overlapping runs
 * with futures. */
hxc_status hxc_varcoef_adjoint_run(hxc_device dev, hxc_buffer u0, hxc_buffer kappa,
                                   hxc_buffer lamT, int64_t ny, int64_t nx, double c, int steps,
                                   int every, hxc_mode mode, hxc_buffer gk, hxc_buffer gu0,
                                   hxc_buffer uT, const hxc_future *deps, int ndeps,
                                   hxc_future *out, hxc_run_stats *stats);
/* Forward only: `steps` variable-diffusivity steps of u0 into uT (one
 * problem; coefficients computed once; uT must not alias u0 or kappa). */
hxc_status hxc_varcoef_forward_run(hxc_device dev, hxc_buffer u0, hxc_buffer kappa, int64_t ny,
                                   int64_t nx, double c, int steps, hxc_buffer uT,
                                   const hxc_future *deps, int ndeps, hxc_future *out,
                                   hxc_run_stats *stats);

/* Checkpoint tapes (the paper has no counterpart; the forward pass of a
 * training step keeps what its backward pass needs, as reverse-mode
 * differentiation does).  A tape for `steps` steps checkpointed every
 * `every` steps (0: ceil(sqrt(steps))) holds *states = max(1,
 * ceil(steps / every)) fields of ny x nx doubles, checkpoint k being the
 * state after k * every steps (checkpoint 0 = u0). */
hxc_status hxc_varcoef_tape_states(int steps, int every, int64_t *states);
/* hxc_varcoef_forward_run that also writes the tape (at least *states * ny
 * * nx * 8 bytes; it must not overlap u0, kappa or uT).  The states are
 * computed by the same kernels in the same order as the forward pass of
 * hxc_varcoef_adjoint_run, so the two give the same bits. */
hxc_status hxc_varcoef_forward_tape(hxc_device dev, hxc_buffer u0, hxc_buffer kappa, int64_t ny,
                                    int64_t nx, double c, int steps, int every, hxc_buffer uT,
                                    hxc_buffer tape, const hxc_future *deps, int ndeps,
                                    hxc_future *out, hxc_run_stats *stats);
/* hxc_varcoef_adjoint_run from a tape written by hxc_varcoef_forward_tape
 * with the same kappa, c, steps and every: no forward pass, only the
 * segment recomputations and the adjoint steps.  Results bit-identical to
 * hxc_varcoef_adjoint_run's; the tape is read only. */
hxc_status hxc_varcoef_adjoint_tape(hxc_device dev, hxc_buffer tape, hxc_buffer kappa,
                                    hxc_buffer lamT, int64_t ny, int64_t nx, double c, int steps,
                                    int every, hxc_mode mode, hxc_buffer gk, hxc_buffer gu0,
                                    const hxc_future *deps, int ndeps, hxc_future *out,
                                    hxc_run_stats *stats);

/* ------------------------------------------------------------ tuning */

/* Launch-shape and work-split knobs of the built-in kernels (the
 * autotuner's parameters).  They change speed only: every value gives
 * bit-identical results.  Values are clamped to their ranges.  Keys:
 *   "heat2d.emul"  share of the 2D stencil's two FP64 additions per point
 *                  (its pair sum and the sum of its two pair sums) computed
 *                  by the integer-pipe IEEE adder instead of the FP64 pipe,
 *                  in half-additions per point, 0..4 (default 0).
 *   "heat2d.rows"  rows each warp of the 2D kernel walks (default 16).
 *   "heat2d.occupancy"  minimum resident 256-thread CTAs per SM the 2D
 *                  kernel is compiled for, 4..6 (default 4).
 *   "heat3d.zchunks"  z chunks of a 3D launch of form 2, 0 = fill whole
 *                  waves.
 *   "heat3d.variant"  3D kernel form: 2 = three plane registers per level
 *                  (rotated, z loop unrolled by 3), arithmetic on paired FP32
 *                  instructions, 64 x 32 regions, z cut into chunks (also
 *                  the form for planes of more than 2^32 cells), 3 = two
 *                  plane registers per level (centre + partial sum), 2 x 4
 *                  cells per thread, 64 x 64 regions, the z range split
 *                  evenly over one CTA per SM, 4 = form 3 with the input
 *                  planes copied into a shared-memory ring two planes ahead,
 *                  6 = form 4 with packed narrow tiles (the columns and rows
 *                  left over by the 64 - 2T wide output tiles go to 16-wide
 *                  regions run four or sixteen to a CTA in lane segments and
 *                  warp groups; the default), 7 = form 6 with the input
 *                  planes of the regions that lie inside the field (no
 *                  periodic wrap; 4 steps per launch, nx % 4 == 0) copied by
 *                  TMA tensor copies completing on shared-memory barriers
 *                  (bounded waits, see hxc_debug_wait_errors).  Forms 3, 4, 6
 *                  and 7 launched with an hxc_launch_cfg take 512 threads per
 *                  CTA and any grid (forms 6 and 7 at least one CTA per kind
 *                  of tile they have).
 *   "heat3d.variant1"  the form used for one-step launches (PLAIN mode and
 *                  single-step remainders), the values above plus 5 = a
 *                  streaming kernel (4 adjacent x cells per thread, 16-byte
 *                  loads, 64-plane z chunks; nx % 4 == 0 and 16-byte aligned
 *                  fields without a launch cfg, else form 3), the default.
 *   "heat1d.tb_ctas"  CTAs per partition of the temporally blocked 1D
 *                  kernel, 0 = SMs / partitions.
 *   "heat1d.steps_per_launch"  steps per fused 1D launch when the caller
 *                  passes 0, 0..1024 (default 0 = all steps in one launch).
 *   "heat3d.steps_per_launch"  steps per fused 3D launch when the caller
 *                  passes 0, 1..4 (default 4).
 *   "mandel.pair"  Mandelbrot kernel form: 1 = two horizontally adjacent
 *                  pixels per thread on paired FP32 instructions (default),
 *                  0 = one pixel per thread.
 *   "batch.ctas_per_sm"  CTAs per SM of the persistent batch kernel (4).
 *   "batch.block"  threads per CTA of the persistent batch kernel: 256 (default),
 *                  512 or 1024; blocks x CTAs per SM must fit the SM.
 *   "batch.smem_side"  the persistent batch kernel keeps both fields of a
 *                  problem of side <= this value in shared memory for the
 *                  whole run (2 side^2 doubles per CTA), 0..119 (default 0:
 *                  none).
 * Returns HXC_E_INVALID for an unknown key. */
hxc_status hxc_tune_set(const char *key, int64_t value);
hxc_status hxc_tune_get(const char *key, int64_t *value);
/* Loads a tuning cache written by the autotuner: a JSON object
 * {"sm_<major><minor>": {"key": integer, ...}, ...} (the entry of the given
 * architecture is applied; unknown keys are ignored).  The first
 * hxc_get_all_devices call loads HXC_TUNE_CACHE, or tune_cache.json next to
 * the library, automatically. */
hxc_status hxc_tune_load(const char *path, int major, int minor);

/* ------------------------------------------------------- diagnostics */

/* Arithmetic pipes hxc_pipe_rate can measure. */
#define HXC_PIPE_F64_FMA 0 /* FP64 fused multiply-add */
#define HXC_PIPE_F64_ADD 1 /* FP64 add                */
#define HXC_PIPE_F32_FMA 2 /* FP32 fused multiply-add */

/* The paper has no counterpart to this call.  Measured throughput of one
 * arithmetic pipe of the device, the denominator of the rooflines of
 * arithmetic-bound kernels (the FP64 stencils here are bound by the FP64
 * pipe, not by memory).  A kernel of independent dependency chains that
 * issues only the measured instruction (8 chains per thread, 8 CTAs of 256
 * threads per SM) runs once to warm up and once timed with CUDA events
 * (about 0.1 s on B300).  *ops_per_s: operations per second, a fused
 * multiply-add counting as one; *sm_mhz (may be NULL): the SM clock during
 * the timed launch, from the first CTA's clock64 ticks over globaltimer
 * nanoseconds.  Synchronous; allocates and frees a few MB of device memory
 * and a private stream.  HXC_E_INVALID for an unknown kind. */
hxc_status hxc_pipe_rate(hxc_device dev, int kind, double *ops_per_s, double *sm_mhz);

/* ------------------------------------------- norms without allocation */

/* Largest tile grid (tiles_y * tiles_x) hxc_tile_norms_noalloc accepts. */
#define HXC_NOALLOC_MAX_TILES 256

/* The paper has no counterpart to this call.  Per-tile L2 norms
 * sqrt(sum u^2) of a row-major ny x nx field of doubles cut into a
 * tiles_y x tiles_x grid (rows split at p*ny/tiles_y; columns at
 * 2*(q*(nx/2)/tiles_x) when nx is even, else q*nx/tiles_x -- the tiles of
 * hxc_heat2d_run), written to norms[p*tiles_x + q], with the same fixed
 * reduction order (and so the same bits) as HXC_K_TILE_NORM2.
 *
 * It allocates nothing, for callers that must not let the library allocate
 * device memory: a time-critical loop in which cudaMalloc would synchronise
 * the device, a process whose device memory belongs to another allocator,
 * or a deployment that forbids allocation after start-up.  Its reduction
 * scratch is a fixed array of about 132 KB compiled into the library and
 * held on every GPU that loads it until the process exits; grids of more
 * than HXC_NOALLOC_MAX_TILES tiles are rejected with HXC_E_INVALID.
 *
 * src and norms are device pointers on the current device, stream a
 * cudaStream_t (NULL: the legacy default stream); the call is asynchronous
 * on that stream and returns launch errors only.  Every call looks up the
 * scratch array's device address (cudaGetSymbolAddress) with the current
 * device, so the address follows device switches and device resets; the
 * first call in a process may load the library's device code for that
 * device, so make it before any stream capture.  Every call on a device
 * shares the one array and clears the counters it needs; calls whose
 * executions overlap on the GPU (different streams, no ordering) race on
 * it and must be serialised by the caller. */
hxc_status hxc_tile_norms_noalloc(const double *src, int64_t ny, int64_t nx, int64_t tiles_y,
                                  int64_t tiles_x, double *norms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HXC_H */
