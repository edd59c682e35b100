/*
 * qdpg -- lattice-wide Gaussian smearing and hadron contractions on GB300.
 *
 * C ABI of libqdpg.so.  The operations are the data-parallel stages that
 * Winter, "Accelerating QDP++/Chroma on GPUs" (Lattice 2011), moves from the
 * host to the GPU: source creation, source/sink smearing and the hadron
 * spectrum (Sec. 5, Fig. 4), expressed on QDP++-style lattice-wide fields
 * (Sec. 1: data-parallel types over the whole lattice).
 *
 * General rules
 * -------------
 *  - Every call returns a qdpg_status (0 = OK).  On failure the thread-local
 *    message is available from qdpg_last_error().  No C++ exception crosses
 *    this interface.
 *  - Device memory is owned by the caller (PyTorch in the Python binding).
 *    The library never frees caller memory.  A qdpg_field_t only BORROWS the
 *    device pointer it wraps.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous with respect to the host unless stated.
 *  - Pointers documented as "device" must be device (or managed) memory of
 *    the current CUDA device; passing host memory is undefined.
 *
 * Lattice and device layout
 * -------------------------
 *  A lattice has extents dims[0..3] (x0 fastest in the canonical site order)
 *  and a decay direction j_decay (the "time" direction, 0..3).  On the
 *  device every field is stored timeslice-major, component-major,
 *  site-fastest ("SoA"):
 *
 *      element(t, comp, s3) at index (t * ncomp + comp) * V3 + s3
 *
 *  where t = x[j_decay], s3 is the lexicographic index of the other three
 *  coordinates (increasing direction order, first one fastest) and V3 is
 *  their product.  An element is one complex number: float2 (QDPG_F32) or a
 *  pair of bfloat16 (QDPG_BF16, real part first).
 *
 *  Components per site (ncomp):
 *    QDPG_COLOR_MATRIX  9    comp = a*3 + b                     (U[a][b])
 *    QDPG_GAUGE        36    comp = mu*9 + a*3 + b              (U_mu[a][b])
 *      reconstruct-12  24    comp = mu*6 + a*3 + b, a in {0,1}  (row 2 = (row0 x row1)^*)
 *    QDPG_FERMION      12    comp = s*3 + c
 *    QDPG_PROPAGATOR  144    comp = (s*3 + c)*12 + (s'*3 + c')  (sink s,c; source s',c')
 *
 *  QDPG_F16 propagators (the reduced-precision storage of the smearing and
 *  contraction path) are stored site-major instead, so that the tensor-core
 *  smearing kernel reads each site's colour vectors contiguously.  With
 *  v = s*12 + s'*3 + c' (the 48 colour vectors of a site) and c the sink
 *  colour, the float16 pair of (t, comp, s3) is word
 *
 *      ((t*3 + v/16) * V3 + s3) * 48 + (v%16)*3 + c
 *
 *  (three groups of 16 vectors, each group site-major).
 *
 *  Scale record.  Every propagator and fermion field (any precision)
 *  represents stored numbers times 2^exp, where exp is a per-field scale:
 *  smearing grows a field by up to (1 + 6 kappa) per iteration, far beyond
 *  the float16 range and, after squaring in the contractions, beyond FP32.
 *  exp (and, for float16, the largest stored magnitude) lives in a scale
 *  record of QDPG_SCALE_RECORD_BYTES bytes placed after the data, at byte
 *  offset round_up(V*ncomp*esize, 256); the record is part of the field
 *  (qdpg_field_bytes includes it) and every operation on the field reads or
 *  updates it on the device.  Import and point source set exp = 0 (float16
 *  import: the exponent that fits the data); export multiplies by 2^exp;
 *  the contractions apply it to their FP64 sums.  Float16 propagators are
 *  rescaled every iteration; FP32/BF16 fields only when the growth bound of
 *  a smearing call, N log2(1 + 6|kappa|), exceeds 40 bits.  Gauge fields
 *  need no scale (|U_ab| <= 1); F16 links use the component-major layout.
 *
 *  Canonical layout (import/export): complex numbers, site index
 *  x0 + L0*(x1 + L1*(x2 + L2*x3)); propagator/fermion/colour matrix are
 *  [site][comp] with the comp order above; the gauge field is
 *  [mu][site][a][b].
 */
#ifndef QDPG_H
#define QDPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qdpg_lattice* qdpg_lattice_t; /* opaque, owned by the library */
typedef struct qdpg_field* qdpg_field_t;     /* opaque header, data borrowed */

typedef enum {
  QDPG_OK = 0,
  QDPG_ERR_ARG = -1,         /* null pointer, value out of range */
  QDPG_ERR_SHAPE = -2,       /* fields on different lattices, wrong kind, buffer too small */
  QDPG_ERR_DTYPE = -3,       /* precision not valid for this kind or operation */
  QDPG_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed */
  QDPG_ERR_NOMEM = -5,       /* a host or device allocation failed */
  QDPG_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
  QDPG_ERR_UNSUPPORTED = -7  /* valid request this build does not implement */
} qdpg_status;

typedef enum {
  QDPG_COLOR_MATRIX = 0,
  QDPG_GAUGE = 1,
  QDPG_FERMION = 2,
  QDPG_PROPAGATOR = 3
} qdpg_kind;

typedef enum {
  QDPG_F32 = 0,       /* complex float32 (float2) */
  QDPG_BF16 = 1,      /* complex bfloat16 pair (see the accuracy note below) */
  QDPG_F32_R12 = 2,   /* gauge only: float2, two rows stored */
  QDPG_BF16_R12 = 3,  /* gauge only: bfloat16 pair, two rows stored */
  QDPG_F16 = 4,       /* complex float16 pair; propagator or gauge (layout notes above) */
  QDPG_F16_R12 = 5    /* gauge only: float16 pair, two rows stored */
} qdpg_prec;

/* Accuracy of the reduced-precision storages (measured against the FP32
 * path, which agrees with an FP64 computation to ~1e-6):
 *  - QDPG_F16 propagators with F16 / F16_R12 links (per-field power-of-two
 *    scale, tensor-core hop): zero-momentum meson correlators within 4e-3 on
 *    uneven smearing jobs with N up to 50 and kappa up to 0.30, and within
 *    2.5e-3 on the 48^3x96 workload (N up to 80): inside a 2e-2 bound;
 *  - QDPG_BF16 propagators with BF16 reconstruct-12 links: 1-2% on the
 *    24^3x48 workload (N = 40, kappa = 0.21), but up to 3.2e-2 on uneven jobs
 *    of the same N and kappa range, already 1% at N = 5 (the 8-bit links
 *    dominate): BF16 storage does NOT hold a 2e-2 bound in general; use F16
 *    storage where that bound must hold. */

/* Size of the scale record of a propagator or fermion (see the layout
 * notes): int32 exp, float max |stored|, then the per-iteration scale slots
 * of a float16 smearing call (at most QDPG_F16_MAX_ITER iterations). */
#define QDPG_SCALE_RECORD_BYTES 8192
#define QDPG_F16_MAX_ITER 999

typedef enum {
  QDPG_CANON_F64 = 0, /* canonical buffer of complex double (2 x double) */
  QDPG_CANON_F32 = 1  /* canonical buffer of complex float  (2 x float)  */
} qdpg_canon;

/* Library version, major*10000 + minor*100 + patch. */
int qdpg_version(void);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t qdpg_launch_count(void);

/* Copy the calling thread's last error message into buf (always
 * NUL-terminated when n > 0).  Returns the status of the failed call, or
 * QDPG_OK if none failed. */
int qdpg_last_error(char* buf, size_t n);

/* ---- kernel timing ------------------------------------------------------
 * When enabled, each kernel the library launches is bracketed by two CUDA
 * events recorded on its own stream.  Kernel names: "smear_hop",
 * "smear_hop_f16", "meson_2pt", "baryon_2pt", "momentum_project", "field_import",
 * "field_export", "shift", "point_source".
 * query() waits for the recorded events and returns the summed elapsed time
 * (ms) and launch count for one name since the last reset().  At most 65536
 * launches are recorded per window.  Host-side bookkeeping is thread-safe. */
int qdpg_profile_enable(int on);
int qdpg_profile_reset(void);
int qdpg_profile_query(const char* name, double* total_ms, uint64_t* launches);

/* ---- device status of bounded waits ---------------------------------------
 * Pipelined kernels wait on shared-memory barriers with a time limit (1 s by
 * default).  A wait that runs out does not trap: the kernel records a flag in
 * a per-device status word, finishes its own in-flight copies and returns.
 * qdpg_device_status synchronises `stream`, reads and clears that word, and
 * returns QDPG_ERR_TIMEOUT if any flag was set (QDPG_OK otherwise). */
int qdpg_device_status(void* stream);

/* Test hooks for the failure path above (host-side settings, process-wide):
 *  QDPG_DEBUG_WAIT_TIMEOUT_NS  time limit of every bounded wait, 1e3..6e10 ns;
 *  QDPG_DEBUG_DROP_STAGE       pipeline stage (counted from 0 within each
 *                              CTA of the pipelined smearing kernel) whose
 *                              copies are skipped, so that the waits for it
 *                              run out; -1 (default) = none;
 *  QDPG_DEBUG_FORCE_SIMPLE_HOP nonzero: always use the one-thread-per-site
 *                              smearing kernel without the copy pipeline;
 *  QDPG_DEBUG_FAIL_ALLOCS      the next `value` device allocations of the library's
 *                              temporaries fail as if the device were out of memory
 *                              (the calls return QDPG_ERR_NOMEM); 0 = none;
 *  QDPG_DEBUG_STAGE_BYTES      largest chunk (bytes of canonical data, at least one
 *                              timeslice) of the host-buffer import/export; 0 = 256 MiB;
 *  QDPG_DEBUG_MESON_FORM       kernel of the F32/BF16 meson contractions: 0 (default) the
 *                              best that applies (the orbit kernel where every channel's
 *                              two masks are equal, as for the sixteen mesons), 1 the
 *                              kernel that stages S2 in shared memory, 2 the kernel that
 *                              reads both propagators from global memory (the forms agree
 *                              to FP32 rounding);
 * and launch-shape settings of the pipelined smearing kernel:
 *  QDPG_TUNE_TILE_CONSUMERS    most sites (threads) per tile, 32..288, 0 = default;
 *  QDPG_TUNE_STAGES            pipeline depth 2..16, 0 = as many as fit (0);
 *  QDPG_TUNE_GRID              0: persistent CTAs (default), 1: one CTA per item;
 * and of the float16 (tensor-core) smearing kernel:
 *  QDPG_TUNE_F16_WARPS         consumer warps per CTA, 8 or 16 (0 = default, 16);
 *  QDPG_TUNE_TENSOR_COPY       FP32/BF16 pipelined hop: 0 (default) stages whole-plane
 *                              tiles with one tensor-map (TMA) copy per stage where
 *                              planes z-1..z+1 are consecutive, and halo tiles of the
 *                              fixed shapes (x extent 16, 24, 48) row-major with five
 *                              tensor-map copies per stage; 1 uses bulk copies only
 *                              (the same results bit for bit). */
enum {
  QDPG_DEBUG_WAIT_TIMEOUT_NS = 1,
  QDPG_DEBUG_DROP_STAGE = 2,
  QDPG_DEBUG_FORCE_SIMPLE_HOP = 3,
  QDPG_TUNE_TILE_CONSUMERS = 4,
  QDPG_TUNE_STAGES = 5,
  QDPG_TUNE_GRID = 7,
  QDPG_TUNE_F16_WARPS = 8,
  QDPG_TUNE_TENSOR_COPY = 9,
  QDPG_DEBUG_FAIL_ALLOCS = 11,
  QDPG_DEBUG_STAGE_BYTES = 12,
  QDPG_DEBUG_MESON_FORM = 13
};
int qdpg_debug_set(int what, long long value);

/* Device allocations the library has made for its own temporaries in this
 * process (smearing scratch when none is given, site values of the momentum
 * projection, staging buffers of the host-buffer import/export).  All are
 * stream-ordered, from the library's own memory pool on each device
 * (cudaMallocFromPoolAsync; created on first use, it keeps up to 4 GiB of
 * freed memory mapped for the next call), and freed on the same stream.
 * qdpg_device_pool_used reports the bytes of that pool in use on the current
 * device. */
uint64_t qdpg_device_alloc_count(void);
int qdpg_device_pool_used(uint64_t* bytes);

/* ---- autotuning of the smearing kernel --------------------------------------
 * The pipelined smearing kernel's tile width and grid (persistent or one CTA
 * per work item) are picked per (lattice, j_decay, psi precision, link
 * precision) by measurement.  qdpg_tune_smear times each candidate with
 * `reps` hops from psi into scratch on `stream` (psi is read, never written;
 * scratch is overwritten) and stores the fastest in a process-wide table that
 * later qdpg_gauss_smear calls on such fields use.  It synchronises the host
 * with the stream.  QDPG_ERR_UNSUPPORTED if the pipelined kernel does not
 * serve the geometry (then the one-thread-per-site kernel is used anyway).
 * Explicit QDPG_TUNE_* settings take precedence over the table.
 * qdpg_tune_query reports the stored choice (sites per tile, grid mode, and
 * measured microseconds per hop); qdpg_tune_save / qdpg_tune_load write and
 * read the table as text, one configuration per line. */
int qdpg_tune_smear(qdpg_field_t U, qdpg_field_t psi, qdpg_field_t scratch, int j_decay, int reps, void* stream);
int qdpg_tune_query(qdpg_field_t U, qdpg_field_t psi, int* consumers, int* grid_mode, float* us_per_hop);
int qdpg_tune_save(const char* path);
int qdpg_tune_load(const char* path);

/* ---- lattice geometry (paper Sec. 1: QDP++ lattice-wide types) ---------- */

/* Create a lattice of extents dims[4] (each >= 1, product < 2^31, at most
 * 65535 timeslices) with decay direction j_decay in 0..3.  *out is owned by
 * the library until qdpg_lattice_destroy.  Host-only; no CUDA call. */
int qdpg_lattice_create(const int dims[4], int j_decay, qdpg_lattice_t* out);
void qdpg_lattice_destroy(qdpg_lattice_t lat);

/* Bytes a field of (kind, prec) needs on this lattice (0 if invalid). */
size_t qdpg_field_bytes(qdpg_lattice_t lat, int kind, int prec);

/* Wrap caller-owned device memory (>= qdpg_field_bytes, 16-byte aligned) as
 * a field.  No copy, no allocation on the device.  The field keeps its own
 * copy of the geometry, so it stays valid after the lattice is destroyed. */
int qdpg_field_wrap(qdpg_lattice_t lat, int kind, int prec, void* dev_ptr, size_t bytes,
                    qdpg_field_t* out);
void qdpg_field_release(qdpg_field_t f);

/* ---- field setup (paper Sec. 5: source creation) ------------------------- */

/* Convert a canonical-layout buffer (device memory, element type `canon`)
 * into `dst`'s device layout and precision.  F32 storage rounds to nearest
 * even; BF16 rounds to nearest even from the value given; reconstruct-12
 * keeps rows 0 and 1.  F16 propagators first find the largest |re|, |im|
 * (M), set exp = e - 14 where M = f 2^e with f in [0.5, 1), and store the
 * values times 2^-exp rounded to nearest even (two kernels); F16 links are
 * rounded directly.  The source must hold V*ncomp complex numbers (gauge:
 * 4*V*9). */
int qdpg_field_import(qdpg_field_t dst, const void* canon_dev, int canon, void* stream);

/* Write `src` to a canonical complex-double buffer in device memory
 * (reconstruct-12 gauge fields are expanded to all nine entries; F16
 * propagators are multiplied by 2^exp, which is exact). */
int qdpg_field_export(qdpg_field_t src, double* canon_dev, void* stream);

/* Host-buffer forms of import and export (Sec. 5 source creation: the
 * propagator arrives from the host, and the smeared fields and correlators
 * go back to it).  `host_canon` is host memory in the canonical layout
 * above (import: complex double or complex float per `canon`; export:
 * complex double).  Same conversions as qdpg_field_import/export.
 *  - The data moves through a device staging buffer that the library
 *    allocates stream-ordered (the library's pool, see below) and frees on `stream` after
 *    the last chunk: one cudaMemcpyAsync per contiguous run of whole
 *    timeslices (at most 256 MiB of canonical data per chunk) when
 *    j_decay = 3, where a timeslice is contiguous in the canonical order
 *    (four runs per chunk for a gauge field, one per direction); otherwise
 *    the whole field in one chunk.  F16 propagators read the host data
 *    twice (the first pass finds the largest magnitude that fixes the scale).
 *  - Page-locked host memory (cudaHostAlloc / cudaHostRegister) keeps the
 *    calls asynchronous; with pageable memory they are still correct but
 *    the copies synchronise with the host.  The host buffer must stay
 *    valid (import) or untouched (export) until `stream` has passed the call.
 *  - QDPG_ERR_NOMEM if the staging buffer cannot be allocated; QDPG_ERR_CUDA
 *    if a copy fails. */
int qdpg_field_import_host(qdpg_field_t dst, const void* host_canon, int canon, void* stream);
int qdpg_field_export_host(qdpg_field_t src, double* host_canon, void* stream);

/* Point source at x0 (Sec. 5 "source creation"): zero the field, then set
 * the unit entries at x0.  PROPAGATOR: all twelve columns,
 * S[s c][s' c'] = delta_ss' delta_cc'; FERMION: the single entry
 * spin_color = s*3 + c (0..11).  F32, BF16 or (propagators) F16 storage;
 * an F16 propagator's scale becomes exp = 0. */
int qdpg_point_source(qdpg_field_t f, const int x0[4], int spin_color, void* stream);

/* ---- shift (QDP++ nearest-neighbour access, Sec. 1) ---------------------- */

/* dst(x) = src(x + sign*mu_hat), periodic; sign = +1 (FORWARD) or -1.
 * dst and src must be distinct fields of the same kind, precision and
 * lattice.  Bit-exact copy of elements (and of an F16 propagator's scale). */
int qdpg_shift(qdpg_field_t dst, qdpg_field_t src, int sign, int mu, void* stream);

/* ---- Gaussian smearing (Sec. 5: SRC and SNK stages) --------------------- */

/* In-place covariant Gaussian smearing, n_iter iterations of
 *   psi(x) <- psi(x) + kappa * sum_{i != j_decay} [ U_i(x) psi(x+i)
 *                                                  + U_i(x-i)^dag psi(x-i) ]
 * acting on colour; every spin and source column is smeared alike.
 * U: QDPG_GAUGE (F32, F32_R12, BF16_R12 or BF16); psi: FERMION or
 * PROPAGATOR (F32 or BF16), same lattice.  Or: psi an F16 PROPAGATOR with
 * U in F16 or F16_R12 (and only then F16 links), smeared by the tensor-core
 * kernel (float16 products, FP32 sums); it needs j_decay equal to the
 * lattice's decay direction, the first non-decay extent a multiple of 4 and
 * at most 64 (QDPG_ERR_UNSUPPORTED otherwise) and n_iter <=
 * QDPG_F16_MAX_ITER; each iteration rescales the stored numbers by a power
 * of two chosen from the previous iteration's largest magnitude, using the
 * scale slots of psi's record.  Arithmetic is FP32 for every storage
 * precision.  j_decay selects the direction that is NOT smeared.
 * scratch: a field of psi's kind/precision/lattice used as the ping-pong
 * buffer; if NULL the library allocates one stream-ordered
 * (cudaMallocAsync) and frees it after the last iteration.  n_iter = 0 is a
 * no-op.  psi and scratch must not alias. */
int qdpg_gauss_smear(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay,
                     qdpg_field_t scratch, void* stream);

/* Gaussian smearing that allocates nothing.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory at the
 * moment they smear -- an application whose own pool manager owns all device
 * memory, code that must not pay the implicit device synchronisation of
 * cudaMalloc/cudaFree, or a process whose memory budget is fixed up front.
 * Same operation, arguments and errors as qdpg_gauss_smear minus `scratch`:
 * the ping-pong buffer is a static device array owned by the library,
 * 32 MiB (33554432 bytes), held on every GPU that loads the library until
 * the process exits.  A psi field larger than that returns QDPG_ERR_ARG
 * before any launch.  No cudaMalloc, cudaFree or other allocating routine
 * is called.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * contents behind (each call overwrites it before reading it); calls whose
 * work overlaps on the GPU -- other streams, other host threads -- race on
 * it, so the caller must serialise them. */
int qdpg_gauss_smear_noalloc(qdpg_field_t U, qdpg_field_t psi, double kappa, int n_iter, int j_decay,
                             void* stream);

/* ---- meson two-point functions (Sec. 5: HAD, mesonic) ------------------ */

/* For channels j = 0..n_chan-1 and momenta k = 0..n_mom-1:
 *   out[j][k][t] = sum_{x: x[j_decay]=t} exp(-i p_k.(x - origin))
 *                  tr[ Gamma(gamma_snk[j]) S1(x) Gamma(gamma_src[j])^dag
 *                      gamma_5 S2(x)^dag gamma_5 ]
 * Gamma(n) = g1^n0 g2^n1 g3^n2 g4^n3 in the DeGrand-Rossi basis (n in 0..15,
 * Gamma(15) = gamma_5), p_k = 2 pi (moms[3k]/L_a, moms[3k+1]/L_b,
 * moms[3k+2]/L_c) over the three non-decay directions a < b < c.
 * S1, S2: PROPAGATOR fields (F32, BF16 or F16, both the same) on the same
 * lattice (may be the same field); F16 sums are multiplied by
 * 2^(exp1 + exp2).  origin: 4 ints or NULL (= 0).
 * out_dev: device buffer of n_chan*n_mom*Nt complex doubles (2 doubles,
 * re then im), overwritten.  Site products are FP32; timeslice and momentum
 * sums are FP64.  Limits: n_chan <= 256, n_mom <= 64. */
int qdpg_meson_2pt(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src,
                   int n_chan, const int* moms, int n_mom, const int origin[4], double* out_dev,
                   void* stream);

/* All ordered pairs of a set of propagators in one pass (Sec. 5: the hadron
 * spectrum of many smeared sources and sinks at once):
 *   out[a][b][j][k][t] = the qdpg_meson_2pt value of S1 = props[a],
 *                        S2 = props[b], channel j, momentum k, timeslice t
 * for a, b = 0..n_props-1.  Every site of every propagator is read once for
 * all n_props^2 pairs (an F32 48^3x96 propagator is 12.2 GB: 8 of them read
 * once instead of 64 pairwise reads of two each).  The per-site traces of all
 * pairs and channels go, a batch of timeslices at a time (at most 4 GiB of
 * site values), to a library buffer and are projected on the tensor cores
 * (qdpg_momentum_project), each pair's sums multiplied by 2^(exp_a + exp_b).
 * props: 1..8 PROPAGATOR fields, all F32, all BF16 or all F16, same lattice.
 * Channels: 1..16, each with Gamma_snk and Gamma_src that permute spin alike
 * (true for Gamma_snk = Gamma_src, as for the sixteen mesons; others return
 * QDPG_ERR_UNSUPPORTED).  moms, n_mom, origin as in qdpg_meson_2pt.
 * out_dev: device buffer of n_props^2*n_chan*n_mom*Nt complex doubles,
 * overwritten.  QDPG_ERR_NOMEM if the library's buffers cannot be allocated. */
int qdpg_meson_2pt_multi(const qdpg_field_t* props, int n_props, const int* gamma_snk, const int* gamma_src,
                         int n_chan, const int* moms, int n_mom, const int origin[4], double* out_dev,
                         void* stream);

/* ---- baryon two-point functions (Sec. 5: HAD, baryonic) ----------------- */

/* For momenta k = 0..n_mom-1:
 *   out[k][t] = sum_{x: x[j_decay]=t} exp(-i p_k.(x - origin))
 *               sum_{alpha alpha'} P_{alpha' alpha} < chi_alpha(x) chibar_alpha'(origin) >
 * with P = (1 + parity * gamma_4)/2 and, for kind 0 (nucleon, uud),
 * chi = eps_abc (u_a^T C gamma_5 d_b) u_c; for kind 1 (Delta++, uuu),
 * chi = eps_abc (u_a^T C gamma_3 u_b) u_c; C = gamma_2 gamma_4 and
 * chibar = eps_a'b'c' ubar_c' (qbar_b' Gbar qbar_a'^T), Gbar = g4 G^dag g4
 * (DeGrand-Rossi basis).  Every Wick pairing enters with the sign of the
 * Grassmann reordering; the fully nested pairing has sign +1.  Su, Sd:
 * point-to-all PROPAGATOR fields (F32, BF16 or F16, both the same, same
 * lattice; F16 sums are multiplied by 2^(2 exp_u + exp_d)); Sd is used by
 * the nucleon only and may be NULL for the Delta.  origin: 4 ints or NULL;
 * momenta as in qdpg_meson_2pt.  out_dev: device buffer of n_mom*Nt
 * complex doubles, overwritten.  Site values FP32, sums FP64.
 * Limits: n_mom <= 64. */
int qdpg_baryon_2pt(qdpg_field_t Su, qdpg_field_t Sd, int kind, int parity, const int* moms, int n_mom,
                    const int origin[4], double* out_dev, void* stream);

/* ---- site values and momentum projection on the tensor cores ------------- */

/* Site values instead of sums: sites_dev (device, 8-byte aligned) receives
 * complex floats sites[j][t][x3] = the channel-j site trace of
 * qdpg_meson_2pt at the site (t, x3) (device layout order), n_chan*Nt*V3
 * of them (F16 fields: scaled by the power of two in FP32, which can
 * overflow for fields smeared far beyond 2^60). */
int qdpg_meson_sites(qdpg_field_t S1, qdpg_field_t S2, const int* gamma_snk, const int* gamma_src, int n_chan,
                     void* sites_dev, void* stream);

/* As qdpg_baryon_2pt, but writes the site values sites[t][x3] (Nt*V3
 * complex floats) instead of projecting. */
int qdpg_baryon_sites(qdpg_field_t Su, qdpg_field_t Sd, int kind, int parity, void* sites_dev, void* stream);

/* Momentum projection of site values (the dense part of the hadron stage):
 *   out[j][k][t] = sum_{x3} sites[j][t][x3] exp(-i p_k.(x - origin))
 * with sites as written by qdpg_meson_sites / qdpg_baryon_sites on lattice
 * `lat` (n_chan blocks of Nt*V3 complex floats, device memory) and p_k, origin
 * as in qdpg_meson_2pt.  Computed as a complex GEMM on the 5th-generation
 * tensor cores (tcgen05, TF32 with hi/lo operand splitting, FP32
 * accumulation per CTA, FP64 sums across CTAs).  out_dev: device buffer of
 * n_chan*n_mom*Nt complex doubles, overwritten.  Limits: n_mom <= 64. */
int qdpg_momentum_project(qdpg_lattice_t lat, const void* sites_dev, int n_chan, const int* moms, int n_mom,
                          const int origin[4], double* out_dev, void* stream);

/* ---- batches of independent jobs (Sec. 5: many sources at once) ---------- */

/* One job of a batch: smear psi in place (n_iter iterations with kappa,
 * exactly as qdpg_gauss_smear with scratch as the ping-pong buffer) and,
 * if mesons_out is not NULL, then write the sixteen zero-momentum meson
 * correlators of psi with itself (channel j = Gamma(j) at sink and source,
 * as qdpg_meson_2pt with gamma_snk = gamma_src = 0..15, one momentum (0,0,0),
 * origin 0) to mesons_out: a device buffer of 16*Nt complex doubles.
 * The field headers are copied at qdpg_batch_create; the device buffers
 * they point to are borrowed and must outlive the batch. */
typedef struct {
  qdpg_field_t U;       /* QDPG_GAUGE, any link precision */
  qdpg_field_t psi;     /* PROPAGATOR or FERMION, F32 or BF16; or PROPAGATOR F16 (with F16/F16_R12 links) */
  qdpg_field_t scratch; /* same kind/precision/lattice as psi, distinct buffer */
  double kappa;
  int n_iter;           /* >= 0; jobs of one batch may differ */
  double* mesons_out;   /* device, 16*Nt complex doubles, or NULL */
} qdpg_job;

typedef struct qdpg_batch* qdpg_batch_t; /* opaque, owned by the library */

/* Plans a batch of njobs (1..4096) independent jobs; jobs may differ in
 * lattice, precision, kappa and n_iter.  Jobs that share lattice, kind and
 * precisions form one class; each smearing step runs one multi-job launch
 * per class over the jobs whose count is not yet reached (up to 64 jobs per
 * launch).  j_decay: the direction that is not smeared, as in
 * qdpg_gauss_smear.  Errors: QDPG_ERR_ARG for a null pointer, njobs or
 * j_decay out of range, negative n_iter or NaN kappa; QDPG_ERR_SHAPE for
 * fields that do not match; QDPG_ERR_DTYPE for F16 propagators without
 * F16 links or the reverse; QDPG_ERR_UNSUPPORTED for F16 jobs whose
 * j_decay is not the lattice's or whose n_iter exceeds QDPG_F16_MAX_ITER.
 * Float16 jobs run on the tensor-core kernel with their own scale slots.
 * Nothing is launched or allocated on the device. */
int qdpg_batch_create(const qdpg_job* jobs, int njobs, int j_decay, qdpg_batch_t* out);

/* Runs every job of the batch on `stream`.  use_graph = 0: the launches are
 * issued directly.  use_graph = 1: the first such call issues them directly
 * (performing any one-time set-up) and then captures the same sequence into
 * a CUDA graph (thread-local capture mode, on a stream the library creates
 * and destroys for it, so `stream` may be the default stream) without running
 * it again; later calls with use_graph = 1 launch that graph on `stream`.  Every run
 * recomputes from the current contents of the jobs' psi buffers. */
int qdpg_batch_run(qdpg_batch_t batch, int use_graph, void* stream);

/* Frees the plan and its graph.  NULL is a no-op. */
void qdpg_batch_destroy(qdpg_batch_t batch);

#ifdef __cplusplus
}
#endif

#endif /* QDPG_H */
