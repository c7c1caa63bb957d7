/*
 * eri.h -- C ABI of the GB300 engine for batched electron repulsion integrals (ERIs)
 * with fused fixed-bitwidth compression, after arXiv 2303.13632 ("Computing and
 * Compressing Electron Repulsion Integrals on FPGAs").
 *
 * What is computed (paper section in brackets):
 *   [ab|cd] = int int g_a(r) g_b(r) g_c(r') g_d(r') / |r - r'| dr dr'          (Sec. II-B, Eq. 1)
 * for Cartesian Gaussian shells with L <= 4 (s, p, d, f as in Sec. II-A, and g), contracted over
 * primitives, by Rys quadrature (Sec. II-C): Boys function / Rys roots and weights,
 * setup of B and C, vertical recurrence (Eq. 6), horizontal recurrence (Eq. 7) and
 * quadrature (Eq. 8); optionally compressed per quartet into n-bit integers with one
 * scale each (Sec. II-D, Eqs. 9-10; decompression Eq. 11 is the caller's x = q * eps).
 *
 * Conventions shared by every entry point
 *   - Shell functions: N(alpha, L) (x-Ax)^ax (y-Ay)^ay (z-Az)^az exp(-alpha |r-A|^2) with
 *     N = (2 alpha/pi)^{3/4} (4 alpha)^{L/2} / sqrt((2L-1)!!) for every component (the
 *     axis-aligned normalisation of Sec. II-A).  A contracted function is
 *     sum_k coefs[k] N(exps[k], L) g_k; the contraction is not renormalised.
 *   - Cartesian order within a shell: a_x from L down to 0, then a_y from L-a_x down to 0
 *     (xx, xy, xz, yy, yz, zz).  Within a quartet the ERIs are row major: a slowest, d
 *     fastest.  (The FPGA loop order of the paper's Fig. 2 is d, c outer with b, a unrolled;
 *     that is a hardware choice and does not change the values.)
 *   - Class id of a quartet of shells with angular momenta (La, Lb, Lc, Ld):
 *     ((La*4 + Lb)*4 + Lc)*4 + Ld, 0..255, for the 256 generic classes of Sec. III-A (every
 *     L <= 3); 256 + ((La*5 + Lb)*5 + Lc)*5 + Ld for the 369 classes with a g shell (L = 4).
 *     Ids below ERI_NUM_CLASS_IDS that match neither rule (256 + ... with every L <= 3) are not
 *     classes.  Classes with a g shell are computed by one kernel whose angular momenta are
 *     run-time values (the others by kernels specialised per canonical class); their
 *     compressed output goes through a scratch buffer of FP64 values.
 *   - Output order: quartets sorted by class id (ascending), stable within a class (the
 *     order of the caller's list); eri_plan_quartet_order returns the permutation.
 *   - Pointers named d_* are device pointers on the plan's device; every other pointer is
 *     host memory.  The plan owns its device copies; the caller owns every output buffer.
 *   - Calls that take a stream are asynchronous on that stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream).  One plan is used from one stream at a time.
 *   - Errors: no exception crosses the ABI.  Invalid arguments return an error before any
 *     device work and leave outputs untouched.  Device-side problems (non-finite results)
 *     are latched in the plan and returned by eri_sync.
 */
#ifndef GB300_ERI_H
#define GB300_ERI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eri_plan_s *eri_plan_t;

/* Number of class ids (see the class-id rule above): per-class loops run over 0..880. */
#define ERI_NUM_CLASS_IDS 881

typedef enum {
    ERI_OK = 0,
    ERI_E_INVALID = 1,     /* bad argument: null pointer, L < 0, alpha <= 0, non-finite input,
                              shell id out of range, bitwidth outside 2..24, wrong class */
    ERI_E_UNSUPPORTED = 2, /* valid request this build does not serve */
    ERI_E_NOMEM = 3,       /* device or host allocation failed */
    ERI_E_CUDA = 4,        /* a CUDA runtime call failed (launch, copy, sync) */
                           /* 5 is not used: no kernel of this library waits on a flag or a
                              peer, so no bounded wait can give up */
    ERI_E_NUMERIC = 6      /* a non-finite ERI was produced (latched, see eri_sync) */
} eri_status_t;

/* Arithmetic of the recurrence/quadrature stages (Sec. III: the paper uses FP32 there
 * and FP64 for the Rys roots, footnote of Sec. II-C). */
enum {
    ERI_FP64 = 0,  /* everything in FP64 */
    ERI_MIXED = 1  /* FP64: Boys function, Rys roots and weights, Gaussian-product prefactors,
                      B and C (rounded once to FP32); FP32: the 2-D integral recurrences (Eqs.
                      6-7, or for classes with angular momentum on b or d the equivalent
                      four-index recursion, which does not amplify FP32 rounding) and the
                      quadrature (Eq. 8); primitive sums Kahan-compensated */
};

/* How eri_plan_create obtains the quartet list. */
enum {
    ERI_EXPLICIT = 0, /* the caller's list of n_quartets x 4 shell ids */
    ERI_ALL = 1,      /* every ordered quartet (i, j, k, l) of the n_shells shells */
    ERI_UNIQUE8 = 2   /* one quartet per class of the 8-fold permutational symmetry (Sec. II-B,
                         (ij|kl) = (ji|kl) = (ij|lk) = (kl|ij) = ...), enumerated on the device:
                         the unordered shell pairs (i >= j) are ranked by decreasing Schwarz
                         factor Q_ij (ties by increasing i (i+1)/2 + j; all Q are equal without
                         screening), and every pair of ranks r <= s gives the quartet
                         (i_r, j_r, i_s, j_s), listed by r, then s; see schwarz_threshold and
                         shard_count.  `quartets` and n_quartets are ignored. */
};

/* Flags of eri_plan_opts_t.flags */
enum {
    ERI_QUARTETS_ON_DEVICE = 1, /* `quartets` is a device pointer (no host->device copy) */
    ERI_NO_PAIR_TABLE = 2       /* do not build the primitive-pair table (see eri_plan_create) */
};

/* One shell (host memory; eri_plan_create copies it). */
typedef struct {
    double center[3];     /* bohr */
    int32_t L;            /* 0..4 (s, p, d, f, g) */
    int32_t nprim;        /* >= 1 */
    const double *exps;   /* nprim exponents, each > 0 */
    const double *coefs;  /* nprim contraction coefficients (finite) */
} eri_shell_t;

typedef struct {
    int32_t precision;    /* ERI_FP64 or ERI_MIXED */
    int32_t quartet_mode; /* ERI_EXPLICIT, ERI_ALL or ERI_UNIQUE8 */
    int32_t device;       /* CUDA device ordinal the plan lives on */
    int32_t flags;        /* ERI_QUARTETS_ON_DEVICE | ERI_NO_PAIR_TABLE */
    double schwarz_threshold; /* > 0: keep only quartets with Q_ij Q_kl >= threshold, where
                                 Q_ij = sqrt(max |(ab|ab)|) over the components of the pair (the
                                 Cauchy-Schwarz bound |(ij|kl)| <= Q_ij Q_kl), the diagonal ERIs
                                 computed in FP64 by this library's kernels; applies to every
                                 quartet mode.  0 = no screening. */
    int64_t shard_index;  /* ERI_UNIQUE8 only: with shard_count > 1 the plan keeps the quartets */
    int64_t shard_count;  /* at positions shard_index, shard_index + shard_count, ... of the
                             screened enumeration (an even 1-in-shard_count subset, e.g. one
                             replica's share of a job, or a bounded sample of a workload too
                             large to hold).  0 or 1 = all. */
} eri_plan_opts_t;

/* Builds a plan: validates and normalises the shells, classifies and sorts the quartets by
 * class on the device, and keeps device copies of everything the kernels read.  Unless
 * ERI_NO_PAIR_TABLE is set, it also tabulates the Gaussian-product quantities of every pair of
 * primitives (p, 1/p, P - A and the exponential prefactor times both coefficients, 48 bytes a
 * pair, n_prims^2 pairs) when that table stays within 16 GiB and a quarter of the free device
 * memory; the kernels then read them instead of recomputing them per quartet (same values up to
 * rounding order).
 *   shells      n_shells entries (host)
 *   quartets    n_quartets x 4 int32 shell ids, row major (host unless
 *               ERI_QUARTETS_ON_DEVICE), or NULL with ERI_ALL / ERI_UNIQUE8
 *   opts        NULL for defaults (ERI_FP64, ERI_EXPLICIT, device 0, no flags, no screening)
 *   out         receives the plan; untouched on error
 * With a Schwarz threshold the plan first computes the FP64 diagonal ERIs (ij|ij) of all
 * n_shells (n_shells + 1) / 2 pairs (temporary device memory of at most 256 MiB for them, plus
 * the pair-table rule above) and drops the quartets below the threshold before classifying.
 * At most 2^31 - 2 quartets per plan (after screening and sharding).
 * For tests of the error paths, the environment variable ERI_INJECT_NOMEM=k (k >= 1) makes the
 * k-th allocation of each call fail as if memory were exhausted (the host plan object is the
 * first, then the device buffers in program order; the internal plan of diagonal quartets used
 * for screening counts its own allocations the same way): the call then returns ERI_E_NOMEM,
 * frees what it had allocated and leaves *out untouched.
 * Synchronous.  Errors: ERI_E_INVALID (bad shell, id out of range, unknown mode or flag, negative
 * or non-finite threshold, shard_index outside 0..shard_count-1, sharding outside
 * ERI_UNIQUE8), ERI_E_UNSUPPORTED (too many quartets or pairs), ERI_E_NOMEM, ERI_E_CUDA. */
eri_status_t eri_plan_create(const eri_shell_t *shells, int32_t n_shells, const int32_t *quartets,
                             int64_t n_quartets, const eri_plan_opts_t *opts, eri_plan_t *out);

/* Frees the plan and its device memory.  NULL is ignored. */
void eri_plan_destroy(eri_plan_t plan);

/* Moves the plan's shells: replaces the centres, exponents and contraction coefficients of every
 * shell (normalised as in eri_plan_create, Sec. II-A) and rebuilds the primitive-pair table if
 * the plan has one, keeping everything else -- the quartet list and its class order (including
 * the result of any screening, which is not redone), per-class precision, autotuned launch
 * choices and the cached graph of eri_compute_compressed_batched.  This is the per-step call of
 * a geometry loop (molecular dynamics, optimisation): later compute and eri_backward calls see
 * the new shells, with no new plan, host sort or allocation.
 *   shells      n_shells entries (host); n_shells, and every shell's L and nprim, must equal
 *               the plan's
 *   stream      ordered after the plan's earlier work on this stream (cudaStream_t, NULL =
 *               legacy default stream); work of the plan on other streams must have finished
 * Synchronous on `stream` (returns once the new values are on the device).  On ERI_E_INVALID
 * (NULL plan or shells, a changed count, L or nprim, a non-finite centre or coefficient, an
 * exponent <= 0) the plan is unchanged; ERI_E_CUDA from the copies or the table kernel. */
eri_status_t eri_plan_update_shells(eri_plan_t plan, const eri_shell_t *shells, int32_t n_shells,
                                    void *stream);

/* Changes the precision used by later compute calls (ERI_FP64 or ERI_MIXED).  Host only;
 * ERI_E_INVALID for a NULL plan or another value. */
eri_status_t eri_plan_set_precision(eri_plan_t plan, int32_t precision);

/* Precision of one class, overriding the plan's (ERI_FP64, ERI_MIXED, or -1 to follow the plan).
 * Host only (drops the cached graph of eri_compute_compressed_batched); ERI_E_INVALID for a NULL
 * plan, cls not a class id or another value. */
eri_status_t eri_plan_set_class_precision(eri_plan_t plan, int32_t cls, int32_t precision);

/* Chooses the precision of every class of the plan for `bits`-bit output: FP32 recurrences
 * (ERI_MIXED) for the classes whose measured error stays below `max_err_steps` (0 < . <= 1)
 * quantisation steps eps = b_max / (2^{bits-1} - 1), FP64 for the others.  The error of a
 * class is max |mixed - FP64| / b_max over its first `sample` quartets, both computed on the
 * device (quartets with b_max <= 1e-30 Ha are left out), so it is a sample estimate; the
 * decompressed error of a mixed class is then at most eps / 2 (Eq. 10) plus that error.
 * Allocates temporary device buffers; synchronous on `stream`. */
eri_status_t eri_plan_calibrate_precision(eri_plan_t plan, int32_t bits, int64_t sample,
                                          float max_err_steps, void *stream);

/* Effective precision of a class and the error measured by eri_plan_calibrate_precision
 * (-1 when not measured).  Either output may be NULL.  ERI_E_INVALID for a NULL plan or cls
 * outside 0..255. */
eri_status_t eri_plan_class_precision(eri_plan_t plan, int32_t cls, int32_t *precision,
                                      float *mixed_err);

/* Kernel launches eri_compute_class / eri_compute_compressed_class make for class cls in its
 * current precision: 1 for the fused kernels, 2 per chunk of 2^20 quartets (setup and
 * recurrence kernels) on the split path of primitive plans, 0 for an empty class.
 * ERI_E_INVALID for a NULL plan or output, or cls not a class id. */
eri_status_t eri_plan_class_launches(eri_plan_t plan, int32_t cls, int32_t *n_launches);

/* Names of the kernel instantiation(s) eri_compute_compressed_class launches for class cls in
 * its current precision (for reports that group time by kernel, e.g. "eri_setup_kernel<Cfg<2, 1,
 * 1, 0, float>> + eri_class_kernel<Cfg<2, 1, 1, 0, float>, 0, 1>"), NUL-terminated into buf of
 * len bytes.  Host only; ERI_E_INVALID for a NULL plan or buffer, cls not a class id or a buffer
 * too short. */
eri_status_t eri_plan_class_kernels(eri_plan_t plan, int32_t cls, char *buf, size_t len);

/* Total quartets in the plan.  ERI_E_INVALID if either argument is NULL. */
eri_status_t eri_plan_num_quartets(eri_plan_t plan, int64_t *n_quartets);

/* Per-class layout.  cls = ((La*4 + Lb)*4 + Lc)*4 + Ld.  Any output pointer may be NULL.
 *   n_quartets          quartets of this class in the plan
 *   n_eri_per_quartet   n_ga n_gb n_gc n_gd (Sec. II-A shell sizes)
 *   first_quartet       index of the class's first quartet in class-sorted order
 *   fp64_offset         offset (in doubles) of the class's first ERI in eri_compute's output
 * Host only; ERI_E_INVALID for a NULL plan or cls not a class id. */
eri_status_t eri_plan_class_info(eri_plan_t plan, int32_t cls, int64_t *n_quartets,
                                 int32_t *n_eri_per_quartet, int64_t *first_quartet,
                                 int64_t *fp64_offset);

/* perm_out[i] = caller's index of the quartet at class-sorted position i (host array of
 * eri_plan_num_quartets entries).  For ERI_ALL, index = ((i*n + j)*n + k)*n + l; for ERI_UNIQUE8,
 * the quartet's position among the plan's quartets in enumeration order (after screening and
 * sharding).  A screened ERI_EXPLICIT / ERI_ALL plan keeps the index into the unscreened list.
 * Synchronous (reads the plan's device permutation); ERI_E_INVALID for a NULL plan, or a NULL
 * perm_out when the plan has quartets; ERI_E_CUDA if the copy fails. */
eri_status_t eri_plan_quartet_order(eri_plan_t plan, int64_t *perm_out);

/* The plan's quartets (n_quartets x 4 shell ids, host array) in class-sorted order, i.e. the
 * order of every output; the shell order within each quartet is the one the outputs use (for
 * ERI_UNIQUE8 the enumeration's).  Synchronous.  ERI_E_INVALID for a NULL plan, or a NULL
 * quartets_out when the plan has quartets. */
eri_status_t eri_plan_quartets(eri_plan_t plan, int32_t *quartets_out);

/* Quartets before Schwarz screening (for ERI_UNIQUE8: n_pairs (n_pairs + 1) / 2) and quartets
 * that pass it, before sharding (without a threshold the two are equal).  Either output may be
 * NULL.  Host only; ERI_E_INVALID for a NULL plan. */
eri_status_t eri_plan_screening(eri_plan_t plan, int64_t *candidates, int64_t *kept);

/* Sizes of the outputs of eri_compute_compressed for a bitwidth (bits = 0: eri_compute's FP64
 * output).  packed_bytes covers all classes; scales_bytes = 4 * n_quartets.  Host only;
 * ERI_E_INVALID for a NULL plan or bits other than 0 and 2..24.  Either output may be NULL. */
eri_status_t eri_output_bytes(eri_plan_t plan, int32_t bits, size_t *packed_bytes,
                              size_t *scales_bytes);

/* Byte range of one class inside the packed output of eri_compute_compressed.  Each class
 * segment starts on a 256-byte boundary and holds a little-endian, least-significant-bit-
 * first stream of n-bit two's complement fields: ERI v of the class (v = quartet-in-class *
 * n_eri + index-in-quartet) occupies stream bits [v*bits, (v+1)*bits), stream bit s being
 * bit s%32 of 32-bit word s/32.  For bits = 8 and 16 this is a plain int8/int16 array.
 * Bits past the class's last field up to the segment end are zero.  Host only; ERI_E_INVALID
 * for a NULL plan, bits outside 2..24 or cls not a class id.  Either output may be NULL. */
eri_status_t eri_packed_class_offset(eri_plan_t plan, int32_t bits, int32_t cls,
                                     size_t *byte_offset, size_t *bytes);

/* The paper's output layout (Sec. III-C, compress-store loops): each quartet's codes as 512-bit
 * chunks of F = floor(512/bits) n-bit fields, in the quartet's ERI order; the fields that do not
 * fit in a chunk open the next one, and the last chunk of a quartet is zero-padded, so a quartet
 * takes n_CS = ceil(n_eri / F) chunks of 64 bytes and no chunk holds two quartets.  Field j of a
 * chunk occupies chunk bits [j*bits, j*bits + bits), chunk bit s being bit s%32 of the chunk's
 * 32-bit word s/32 (little-endian, least significant bit first, as the dense stream; the paper
 * does not fix the bit order).  Quartets are class-sorted as everywhere else; class segments
 * follow each other without gaps (each is a whole number of chunks).
 * Byte range of class `cls` in that layout; cls = ERI_NUM_CLASS_IDS gives the total size in
 * *byte_offset.
 * bits 2..24; ERI_E_INVALID otherwise.  Host only. */
eri_status_t eri_paper512_class_offset(eri_plan_t plan, int32_t bits, int32_t cls,
                                       size_t *byte_offset, size_t *bytes);

/* Re-lays the packed output of eri_compute_compressed (d_packed, layout of
 * eri_packed_class_offset, read only) into the chunk layout above (d_chunks, written in full:
 * eri_paper512_class_offset(plan, bits, ERI_NUM_CLASS_IDS) bytes).  Integer copy on the GPU, asynchronous on
 * `stream`; both pointers device memory, 4-byte aligned, not overlapping.  The scales are
 * unchanged (one eps per quartet, as written by eri_compute_compressed). */
eri_status_t eri_pack_paper512(eri_plan_t plan, int32_t bits, const void *d_packed, void *d_chunks,
                               void *stream);

/* Same as eri_pack_paper512 for one dense stream without a plan: d_stream holds n_quartets *
 * n_eri n-bit fields, quartet after quartet, as the dense stream above (at least
 * ceil(n_quartets * n_eri * bits / 32) 32-bit words); d_chunks receives n_quartets * n_CS * 64
 * bytes.  n_eri 1..50625, bits 2..24, device pointers 4-byte aligned; ERI_E_INVALID
 * otherwise, ERI_E_CUDA if a launch fails.  n_quartets = 0 does nothing. */
eri_status_t eri_pack_paper512_stream(const void *d_stream, int64_t n_quartets, int32_t n_eri,
                                      int32_t bits, void *d_chunks, void *stream);

/* FP64 ERIs of every quartet (Eqs. 5-8 per primitive quartet, summed over primitives) into
 * d_out (eri_output_bytes(plan, 0, ...) bytes, class-sorted, see fp64_offset).
 * Asynchronous on `stream`; the launches per class are given by eri_plan_class_launches.
 * ERI_E_INVALID for a NULL plan, a NULL d_out when the plan has quartets, or a d_out that is not
 * 8-byte aligned; ERI_E_CUDA if a launch fails.  Non-finite results are latched (eri_sync). */
eri_status_t eri_compute(eri_plan_t plan, double *d_out, void *stream);

/* Same as eri_compute for one class only (cls as in eri_plan_class_info); d_out is the
 * full-size buffer and only the class's range is written. */
eri_status_t eri_compute_class(eri_plan_t plan, int32_t cls, double *d_out, void *stream);

/* ERIs compressed per quartet (Sec. II-D): b_max = max |x| over the quartet, eps = b_max /
 * (2^{bits-1} - 1) rounded to FP32 (Eq. 9, stored 32-bit as in Sec. III-C), q = ANINT(x /
 * eps) with halves away from zero (Eq. 10), computed as x * eps^{-1} like the paper's
 * kernel.  b_max = 0 gives eps = 0 and q = 0.
 *   bits       2..24 (eps has a 24-bit significand; wider codes would exceed +-(2^{n-1}-1))
 *   d_packed   eri_output_bytes(plan, bits, ...).packed bytes, layout of eri_packed_class_offset
 *   d_scales   one float eps per quartet, class-sorted
 * Asynchronous on `stream`.  ERI_E_INVALID for a NULL plan, bits outside 2..24, or NULL or
 * not 4-byte-aligned buffers when the plan has quartets; ERI_E_CUDA if a launch fails. */
eri_status_t eri_compute_compressed(eri_plan_t plan, int32_t bits, void *d_packed, float *d_scales,
                                    void *stream);

/* eri_compute_compressed with the result delivered to host memory: each class's kernels run on
 * `stream`, and as soon as a class finishes its packed segment and scales are copied to the
 * same offsets of h_packed / h_scales on a plan-owned copy stream, overlapping the kernels of
 * the following classes (no counterpart in the paper, whose output crosses PCIe after the run).
 *   d_packed, d_scales  device buffers of eri_output_bytes(plan, bits) sizes (staging)
 *   h_packed, h_scales  host buffers of the same sizes; page-locked memory lets the copies
 *                       overlap the kernels (pageable memory works, serialised)
 * Asynchronous: `stream` completes after the last copy; synchronise it before reading the host
 * buffers.  Errors as eri_compute_compressed. */
eri_status_t eri_compute_compressed_to_host(eri_plan_t plan, int32_t bits, void *d_packed,
                                            float *d_scales, void *h_packed, float *h_scales,
                                            void *stream);

/* eri_compute_compressed for one class only (full-size buffers). */
eri_status_t eri_compute_compressed_class(eri_plan_t plan, int32_t cls, int32_t bits,
                                          void *d_packed, float *d_scales, void *stream);

/* Batched form of eri_compute_compressed (same outputs, same layout): every class of the plan
 * runs as a persistent work-queue kernel (one grid of resident CTAs per class pulling tiles of
 * quartets from an atomic counter, so quartets of uneven contraction degree balance
 * dynamically), the classes spread over four streams forked from `stream`, the whole sequence
 * captured once into a CUDA graph and replayed on later calls with the same bits, precision
 * and output pointers.  The tile counters are plan-owned device memory.  The launch choice per
 * class (kernel family and grid) comes from eri_autotune when it has run.  Classes with a g
 * shell run their plain (non-persistent) launches, all on the first of the four streams since
 * they share the plan's scratch buffer; eri_autotune leaves them out.  Asynchronous. */
eri_status_t eri_compute_compressed_batched(eri_plan_t plan, int32_t bits, void *d_packed,
                                            float *d_scales, void *stream);

/* eri_compute_compressed (same outputs, same layout) as ONE persistent launch of one kernel
 * for every class of the plan: the classes' quartets are cut into tiles (up to 128 quartets of
 * one class) that the resident CTAs pull from a single work queue (an atomic counter), so
 * quartets of uneven class and contraction degree balance across the GPU without per-class
 * launches.  The kernel takes the angular momenta at run time (the kernel of the classes with a
 * g shell, see the class-id rule above): geometry, roots and B, C in FP64 (rounded to FP32 in
 * ERI_MIXED), the four-index Rys recursion and the quadrature in the plan's precision, sums over
 * primitives in FP64; each tile is compressed in the same launch (b_max and eps per quartet,
 * Eq. 9; codes, Eq. 10).  Every class runs in the plan's precision (per-class overrides are not
 * used here).  d_packed is zeroed on `stream` first (tiles OR their shared edge words in); the
 * plan keeps a class table and reuses its scratch buffer.  Codes agree with eri_compute_compressed
 * to +-1 (a different order of the arithmetic for classes without a g shell).  Asynchronous. */
eri_status_t eri_compute_compressed_queue(eri_plan_t plan, int32_t bits, void *d_packed,
                                          float *d_scales, void *stream);

/* Picks, per canonical class of the plan and for the plan's precision and `bits`, the faster
 * persistent launch (thread-per-quartet or shared-memory kernel where both exist; grid of all
 * resident CTAs, one or two CTAs per SM) by timing each candidate on the plan's own quartets
 * (outputs are written to d_packed/d_scales as a side effect).  Choices already recorded for
 * this GPU in the text file cache_path (may be NULL) are reused; new ones are appended.
 * Synchronous on `stream`. */
eri_status_t eri_autotune(eri_plan_t plan, int32_t bits, void *d_packed, float *d_scales,
                          const char *cache_path, void *stream);

/* Adjoint (gradients) of E = sum_q sum_abcd G_q,abcd (ab|cd)_q for an upstream d_G laid out
 * like eri_compute's output (class-sorted, row major per quartet, eri_output_bytes(plan, 0)):
 *   d_dR[3*s + xi]   = dE / d(center[xi] of shell s)          (n_shells x 3, bohr^-1 Ha)
 *   d_dalpha[p]      = dE / d(exponent of primitive p)         (primitives in the order of the
 *                                                               shells' exps arrays)
 * using d g_a/dA_xi = 2 alpha g_{a+1_xi} - a_xi g_{a-1_xi} and d g_a/d alpha =
 * (2L+3)/(4 alpha) g_a - sum_xi g_{a+2_xi} (same coefficient and normalisation N(alpha, L));
 * the Rys recurrences (Eqs. 6-7) are recomputed on index ranges extended by two and
 * contracted with d_G (Eq. 8 with G weights).  Each class runs in its precision (the plan's, or
 * the per-class override): ERI_FP64 in FP64 throughout, for shells with L <= 2 (the extended
 * ranges of f shells exceed the per-CTA shared memory in FP64; such a plan returns
 * ERI_E_UNSUPPORTED before any device work); ERI_MIXED with the 2-D integrals on the extended
 * ranges by the FP32 four-index recursion, G rounded to FP32, the per-thread and per-warp sums
 * in FP32 and the geometry, roots, B and C (rounded once), the sums across warps, primitives and
 * quartets and both outputs in FP64, for every class up to f.  Plans with a g shell return
 * ERI_E_UNSUPPORTED.  Both outputs are zeroed and then accumulated on `stream` (device atomics:
 * summation order, hence the last bits, can vary between runs). */
eri_status_t eri_backward(eri_plan_t plan, const double *d_G, double *d_dR, double *d_dalpha,
                          void *stream);

/* ---- consumer side: decompression fused with Coulomb/exchange digestion ---- */

/* Flags of eri_digest_jk. */
enum {
    ERI_DIGEST_UNIQUE8 = 1,    /* each quartet stands for its 8-fold symmetric images (Sec. II-B) */
    ERI_DIGEST_ACCUMULATE = 2, /* add to d_J / d_K instead of overwriting them */
    ERI_DIGEST_SYMMETRIC = 4   /* with ERI_DIGEST_UNIQUE8 only: the caller's D is symmetric (as an
                                  SCF density is).  The 8-fold images of every quartet then give
                                  each pair of transposed J / K entries equal totals, so half the
                                  sums and half the device atomics are made and the matrices are
                                  symmetrised at the end, J = (J + J^T) / 2 (with
                                  ERI_DIGEST_ACCUMULATE the incoming J, K must be symmetric) */
};

/* Basis functions of the plan: shells in the order given to eri_plan_create, each contributing
 * its (L+1)(L+2)/2 Cartesian components in the order stated at the top of this header, so
 * function index = (sum of the sizes of the earlier shells) + component.  ERI_E_INVALID if
 * either argument is NULL. */
eri_status_t eri_plan_num_basis_functions(eri_plan_t plan, int64_t *n_bf);

/* Coulomb and exchange matrices from the compressed ERIs of the plan, the use for which Sec. I
 * and Sec. II-D store them: each ERI is decompressed as q * eps (Eq. 11) and contracted with the
 * density matrix,
 *     J[mu][nu]  += (mu nu | lam sig) D[lam][sig],      K[mu][lam] += (mu nu | lam sig) D[nu][sig],
 * summed over the plan's quartets.  With ERI_DIGEST_UNIQUE8 every quartet (i j | k l) also
 * contributes through the seven other index permutations under which a real ERI is invariant
 * ((ji|kl), (ij|lk), (ji|lk), (kl|ij), (lk|ij), (kl|ji), (lk|ji); Sec. II-B), each distinct
 * ordered shell quartet once (permutations that map the quartet onto itself, e.g. when i = j,
 * are not repeated), so a plan of the unique quartets (i >= j, k >= l, pair ij >= pair kl)
 * yields the J and K of the full ERI tensor.  Without it each quartet counts once as listed.
 *   bits       2..24, the width d_packed / d_scales were written with
 *   d_packed   output of eri_compute_compressed (or _batched / _to_host's device staging) for
 *              this plan and bits, layout of eri_packed_class_offset
 *   d_scales   one eps per quartet, class-sorted
 *   d_D        n_bf x n_bf FP64, row major (D[lam][sig] at lam * n_bf + sig); need not be
 *              symmetric
 *   d_J, d_K   n_bf x n_bf FP64, row major; overwritten unless ERI_DIGEST_ACCUMULATE
 * Arithmetic: codes times D in FP32 (D is rounded to FP32 once per call; codes up to 24 bits
 * are exact), the sums over the two contracted indices of a quartet in FP32, scaled by eps and
 * added to J and K in FP64 with device atomics (the order of the FP64 additions, hence the last
 * bits, can vary between runs).  The plan keeps an n_bf x n_bf FP32 buffer for the rounded D
 * and a small table of per-class launch parameters (allocated on the first call, the table
 * copied from host memory on `stream` at every call: one launch covers every class).  Asynchronous on `stream`.  ERI_E_INVALID for a NULL plan, bits
 * outside 2..24, unknown flags, ERI_DIGEST_SYMMETRIC without ERI_DIGEST_UNIQUE8, NULL buffers
 * where the plan needs them, or buffers not aligned to their element size; ERI_E_UNSUPPORTED
 * for plans with a g shell; ERI_E_NOMEM / ERI_E_CUDA from allocation or launch failures. */
eri_status_t eri_digest_jk(eri_plan_t plan, int32_t bits, const void *d_packed, const float *d_scales,
                           const double *d_D, double *d_J, double *d_K, int32_t flags, void *stream);

/* ---- no-allocation entry point (no counterpart in the paper) ---- */

/* Largest n_quartets eri_compute_class_noalloc accepts. */
#define ERI_NOALLOC_MAX_QUARTETS 16384

/* FP64 (precision ERI_FP64) or mixed-precision (ERI_MIXED) ERIs of quartets that all belong
 * to generic class `cls` (a class without a g shell: ERI_E_UNSUPPORTED otherwise), written in
 * eri_compute's per-quartet layout (row major, a slowest),
 * for callers that cannot let a library allocate device memory: applications that reserve the
 * device memory themselves and sub-allocate from their own pool, or code that must not risk
 * the synchronisation an allocation call can cause.  This function calls no cudaMalloc,
 * cudaFree or other allocating routine.  Every input and output is caller-owned device memory:
 *   d_cx, d_cy, d_cz   shell centres (n_shells doubles each)
 *   d_pofs, d_nprim    first primitive and primitive count per shell; every shell a quartet
 *                      uses must have nprim = 1 (otherwise bit 2 of *d_err is set and those
 *                      quartets' values are undefined)
 *   d_exps, d_cn       exponent and coefficient times N(alpha, L) per primitive, with
 *                      N = (2 alpha/pi)^{3/4} (4 alpha)^{L/2} / sqrt((2L-1)!!)
 *   d_quartets         n_quartets x 4 int32 shell ids, 16-byte aligned
 *   d_out              n_quartets * n_eri doubles
 *   d_err              one int32, OR-ed with 1 for a non-finite result and 4 for a contracted
 *                      shell (the caller clears it)
 * The only scratch is a file-scope device array of ERI_NOALLOC_MAX_QUARTETS setup records
 * (about 10 MB, resident on every GPU that loads the library until the process exits);
 * n_quartets above the limit returns ERI_E_INVALID before any device work.  Every call
 * shares that array and leaves its contents behind; nothing in it must start at zero (each
 * call writes the records it reads first).  Calls on one device whose device work overlaps
 * (for example on two streams) race on the array: serialise them.  The first call
 * on a device looks up the device addresses of the array and of the library's constant
 * tables (cudaGetSymbolAddress, with that device current) and copies FP32 copies of two table
 * parts from host memory into further file-scope device arrays (about 280 KB; a copy, not an
 * allocation); make that first call before any stream capture.  CUDA loads a library's device
 * code and data lazily by default (CUDA_MODULE_LOADING=LAZY), so the arrays and each class's
 * kernels become resident on their first use, not when the library is loaded: an application
 * that reserves nearly all device memory up front should either make one call per class and
 * precision it will use before that, or run with CUDA_MODULE_LOADING=EAGER.  Asynchronous on
 * `stream` afterwards. */
eri_status_t eri_compute_class_noalloc(int32_t cls, int32_t precision, const double *d_cx,
                                       const double *d_cy, const double *d_cz,
                                       const int32_t *d_pofs, const int32_t *d_nprim,
                                       const double *d_exps, const double *d_cn,
                                       const int32_t *d_quartets, int64_t n_quartets,
                                       double *d_out, int32_t *d_err, void *stream);

/* Waits for the plan's work on `stream` and returns the first latched device error
 * (ERI_E_NUMERIC) or a CUDA error; clears the latch. */
eri_status_t eri_sync(eri_plan_t plan, void *stream);

/* Human-readable name of a status. */
const char *eri_status_string(eri_status_t status);

/* ---- component diagnostics (same device code as the ERI kernels) ---- */

/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt for m = 0..mmax (mmax <= 16), the
 * moments of the Rys weight (Sec. II-C).  d_F[i*(mmax+1) + m] for the n values d_T[i] >= 0. */
eri_status_t eri_boys_device(int32_t mmax, const double *d_T, int64_t n, double *d_F,
                             void *stream);

/* Rys roots x_mu = t_mu^2 and weights w_mu of order nroots (1..9) for each d_T[i] >= 0
 * (the input R_Rys of Sec. II-C, Eq. 5): d_x[i*nroots + mu], d_w[i*nroots + mu], roots in
 * ascending order, sum_mu w_mu x_mu^k = F_k(T) for k < 2*nroots. */
eri_status_t eri_rys_device(int32_t nroots, const double *d_T, int64_t n, double *d_x,
                            double *d_w, void *stream);

/* eri_rys_device as the mixed-precision setup evaluates it (ERI_MIXED, whose roots and weights
 * are rounded to FP32 afterwards): the polynomial terms from the fifth on and the Taylor terms of
 * F_0 / F_1 from the third on in FP32, reciprocals and 1/sqrt from the FP32 approximation with
 * one Newton-Raphson step in FP64; about 1e-9 relative to eri_rys_device.  Same arguments. */
eri_status_t eri_rys_device_mixed(int32_t nroots, const double *d_T, int64_t n, double *d_x,
                                  double *d_w, void *stream);

/* The binary64 -> binary32 -> binary64 conversions the setup stages use (integer arithmetic,
 * IEEE round to nearest, ties to even; no counterpart in the paper): d_f[i] = (float)d_in[i],
 * d_back[i] = (double)d_f[i].  Asynchronous on `stream`. */
eri_status_t eri_convert_device(const double *d_in, int64_t n, float *d_f, double *d_back,
                                void *stream);

/* Fused multiply-add throughput probe (no counterpart in the paper): n_threads threads (a
 * multiple of 256) each run 16 independent chains of 16 * iters FMAs in FP64 (ERI_FP64) or FP32
 * (ERI_MIXED) and store one value each to d_sink (n_threads doubles or floats), so a timed launch
 * does 512 * iters * n_threads floating-point operations: the measured ALU peak the roofline of
 * the FP-bound kernels is quoted against.  Asynchronous on `stream`; ERI_E_INVALID for other
 * arguments. */
eri_status_t eri_fma_probe(int32_t precision, int64_t n_threads, int32_t iters, void *d_sink, void *stream);

/* Class helpers (no device needed). */
int32_t eri_class_id(int32_t La, int32_t Lb, int32_t Lc, int32_t Ld);
/* n_eri = n_ga n_gb n_gc n_gd, n_rys = (La+Lb+Lc+Ld)/2 + 1. */
eri_status_t eri_class_shape(int32_t cls, int32_t *n_eri, int32_t *n_rys);

#ifdef __cplusplus
}
#endif

#endif /* GB300_ERI_H */
