/*
 * gsp.h -- C ABI of the GB300 (sm_103a) library for constant-cost
 * spatio-angular prefiltering of glinty appearance by tensor decomposition
 * (Constant-Cost Spatio-Angular Prefiltering of Glinty Appearance Using Tensor
 * Decomposition, arXiv 2109.14807).
 *
 * The data path:
 *   normal map --gsp_build_footprint_ndfs--> integer NDF histograms of every
 *   2^l x 2^l footprint (Sec. 4.1)
 *   --gsp_cp_decompose--> CP factors of the 5-mode NDF tensor (Sec. 4.2, Eq. 3)
 *   --gsp_build_query_tables--> 1D summed-area tables (Sec. 4.4)
 *   --gsp_range_query--> batched spatio-angular range queries (Sec. 4.4, Eq. 5)
 *   --gsp_range_query_backward--> adjoint of the range query.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are CUDA device pointers, h_* are host pointers.  All
 *    device buffers are allocated and owned by the caller; the library never
 *    allocates device memory and takes scratch space only from a
 *    caller-supplied workspace (d_ws, ws_bytes).
 *  - `stream` is a cudaStream_t passed as an opaque pointer (NULL = legacy
 *    default stream).  Calls enqueue work on `stream` and return without
 *    waiting, except where a comment says the call synchronises.
 *  - Return value: GSP_OK (0) or a negative gsp_status.  Argument errors are
 *    detected on the host before anything is enqueued.  Errors found by the
 *    device (a non-finite normal, a malformed query) are OR-ed into the
 *    caller's 32-bit status word d_status (GSP_DEV_* bits) and never trap.
 *  - Map side N is a power of two, 2 <= N <= 1024 for the NDF build and CP
 *    decomposition (any power of two up to 2^20 for queries); levels <= log2(N) + 1
 *    (level l has 2^l x 2^l footprints, l = 0 .. log2 N); bins B is a power of two,
 *    4 <= B <= 128; rank R is 1 <= R <= 256 for queries and a power of two
 *    8 <= R <= 64 for the CP decomposition (16 <= R for the tensor-core paths).
 *  - NDF tensor layout: int32 / float, C order [l][y][x][s][t]; (s, t) is the
 *    (n.x, n.y) bin; the logical mode order is (x, y, l, s, t).
 *  - Factor matrices are FP32, row-major [rows][R].
 */
#ifndef GSP_H
#define GSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* gsp_stream; /* cudaStream_t */

typedef enum gsp_status {
  GSP_OK = 0,
  GSP_ERR_INVALID_ARG = -1, /* a size, pointer or option is out of range      */
  GSP_ERR_CUDA = -2,        /* a CUDA runtime call failed (see gsp_last_cuda_error) */
  GSP_ERR_WORKSPACE = -3,   /* ws_bytes smaller than the matching *_workspace_bytes */
  GSP_ERR_NONFINITE = -4,   /* non-finite data found (host-visible reports only) */
  GSP_ERR_NUMERIC = -5,     /* a least-squares system could not be solved        */
  GSP_ERR_TIMEOUT = -6,     /* a bounded device wait ran out                     */
  GSP_ERR_UNSUPPORTED = -7  /* feature not available on this device / build      */
} gsp_status;

/* Bits OR-ed into the device status word d_status. */
#define GSP_DEV_NONFINITE_NORMAL 0x1u /* a normal map entry was NaN or Inf     */
#define GSP_DEV_BAD_QUERY 0x2u        /* non-finite field or material >= n_mats */
#define GSP_DEV_NUMERIC 0x4u          /* Gram system not positive definite: the
                                         pseudo-inverse fallback was used      */
#define GSP_DEV_TIMEOUT 0x8u          /* a bounded wait in a kernel gave up    */

#define GSP_MAX_MATERIALS 16
#define GSP_MAX_SWEEPS 512

/* ------------------------------------------------------------------------ */
/* a1 -- binning of the normal map (Sec. 5.2 "binning method")               */
/* ------------------------------------------------------------------------ */

/* Bin every normal of the N x N map.
 *  d_normal_xy: FP32 [N][N][2] = (n.x, n.y), row-major [y][x]; n.z > 0 implied.
 *  d_bins:      uint16 [N][N], written: s * B + t with
 *               s = clamp(floor(fl32(fl32(n.x + 1) * (B/2))), 0, B-1), t from n.y
 *               (FP32, round-to-nearest, no fused multiply-add).
 *  A non-finite normal sets GSP_DEV_NONFINITE_NORMAL and bins to 0. */
int gsp_bin_normals(const float* d_normal_xy, int N, int bins, uint16_t* d_bins,
                    uint32_t* d_status, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* a2 -- exhaustive multi-level footprint histograms (Sec. 4.1)              */
/* ------------------------------------------------------------------------ */

/* Scratch bytes gsp_build_footprint_ndfs needs (the bin map). */
size_t gsp_build_workspace_bytes(int N, int levels, int bins);

/* Integer NDF histogram of every 2^l x 2^l box footprint at every texel, with
 * wraparound (the paper precomputes NDF images of footprints that double in
 * size per level until they cover the map, Sec. 4.1, Fig. 2).  The window of
 * (x, y, l) covers texels ((x - a + i) mod N, (y - a + j) mod N), 0 <= i, j < 2^l,
 * a = floor(2^l / 2).
 *  d_hist: int32 [levels][N][N][B][B] (C order [l][y][x][s][t]), written.
 *  Counts are exact; sum over (s, t) of every footprint is 4^l.
 *  d_hist NULL (implicit form): no histogram is written; the call bins the
 *  map into the first N*N*2 bytes of d_ws (uint16 [N][N] = s * B + t, as
 *  gsp_bin_normals writes it), from which every footprint's histogram is the
 *  box count above.  gsp_cp_prepare and gsp_cp_decompose generate the MTTKRP
 *  operand from the normal map the same way, without the int32 tensor
 *  (L N^2 B^2 x 4 bytes: 47 GB at N = 1024, 11 levels, 32^2 bins).
 *  d_normal_xy NULL or a bad size: GSP_ERR_INVALID_ARG; d_ws smaller than
 *  gsp_build_workspace_bytes(): GSP_ERR_WORKSPACE; both before anything is
 *  enqueued. */
int gsp_build_footprint_ndfs(const float* d_normal_xy, int N, int levels, int bins,
                             int32_t* d_hist, void* d_ws, size_t ws_bytes,
                             uint32_t* d_status, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* a3/a4 -- CP decomposition by ALS (Sec. 4.2, Eq. 3)                        */
/* ------------------------------------------------------------------------ */

typedef enum gsp_precision {
  GSP_PREC_FP32 = 0,    /* MTTKRP with FP32 FFMA on CUDA cores (the plain path)      */
  GSP_PREC_TF32 = 1,    /* tcgen05, TF32 operands, FP32 accumulate; the NDF tensor is
                           one TF32 value, the factor operands TF32 hi + lo pairs     */
  GSP_PREC_BF16 = 2,    /* tcgen05, BF16 operands, FP32 accumulate; the NDF tensor is
                           one BF16 value, the Khatri-Rao operand a BF16 hi + lo pair
                           (two MMAs per K slice, Henry, Tang & Heinecke 2019)      */
  GSP_PREC_BF16_1X = 3, /* tcgen05, both operands rounded once to BF16             */
  GSP_PREC_STRUCTURED = 4, /* exact structured MTTKRP: the tensor is never built.  Each
                           level slice is a box sum of the texel -> bin one-hot
                           (Sec. 4.1), so the footprint window moves onto the spatial
                           factors (its adjoint: alpha_l(u) = sum_{i < 2^l}
                           fx[(u + a - i) mod N]) and every MTTKRP is a pass over the
                           N x N bin map: O(N^2 levels R) FP32 multiply-adds per mode,
                           FP64 for the long sums, instead of the O(N^2 levels B^2 R)
                           contraction; levels <= 11, any N >= 8 of the map limits */
  GSP_PREC_STRUCTURED_GAUSSIAN = 5 /* the same structured MTTKRP for the Gaussian
                           pixel footprint of Eq. geom instead of the box: level l
                           weighs texel u of the footprint at x by g_l(u_x - x)
                           g_l(u_y - y), g_l(d) proportional to exp(-d^2 / (2 s_l^2)),
                           s_l = 1.5 * 2^l / sqrt(12), for |d| <= min(ceil(3 s_l),
                           (N - 1) / 2), normalised to sum 1; T = B^2/4 times the
                           footprint's weight per bin (1 with raw_counts).  Built from
                           d_normal_xy only; ||T||^2 from the exact same-bin
                           autocorrelation of the bin map (O(N^4) integer compares
                           in gsp_cp_prepare: ~0.1 s at N = 1024) */
} gsp_precision;
/* Tensor-core precisions round the NDF tensor without bias: a value between two
 * BF16 (TF32) neighbours goes to the upper one when frac(i * phi) (i = the
 * element's index in [l][y][x][s][t], phi = the golden ratio, 32-bit fixed point)
 * is below its relative distance from the lower one, so representable values,
 * e.g. every count up to 256 (2048), are exact.  Tensor-memory accumulators
 * restart every 16 K steps of the xy pass and every map row of the (l, s, t)
 * pass, and their partial sums are added with round-to-nearest FP32 operations.
 * BF16 needs N >= 64 and TF32 N >= 32 (a K step stays within one map row). */

/* Five factor matrices and the CP weights, device pointers, FP32:
 * fx [N][R], fy [N][R], fl [levels][R], fs [B][R], ft [B][R], lambda [R].
 * The decomposed tensor is sum_r lambda_r fx_r o fy_r o fl_r o fs_r o ft_r. */
typedef struct gsp_cp_factors {
  float* fx;
  float* fy;
  float* fl;
  float* fs;
  float* ft;
  float* lambda;
} gsp_cp_factors;

typedef struct gsp_als_opts {
  int32_t sweeps;    /* sweeps to run (1 .. GSP_MAX_SWEEPS)                       */
  int32_t precision; /* gsp_precision of the MTTKRP operand                       */
  double tol;        /* stop once |fit_k - fit_(k-1)| < tol (Sec. 4.2 uses 1e-4);
                        0 runs exactly `sweeps` sweeps                            */
  int32_t raw_counts;/* 1: decompose the raw counts H instead of the NDF density
                        T = H * B^2 / (4 * 4^l)                                  */
  int32_t reserved;
} gsp_als_opts;

/* Filled by the host after the call when non-NULL (the call then synchronises
 * `stream`).  fit_k = 1 - ||T - T_hat||_F / ||T||_F after sweep k, in FP64. */
typedef struct gsp_als_report {
  int32_t sweeps_done;
  int32_t numeric_fallbacks; /* mode updates that needed the pseudo-inverse */
  double fit[GSP_MAX_SWEEPS];
} gsp_als_report;

/* Workspace bytes for gsp_cp_prepare / gsp_cp_sweeps / gsp_cp_mttkrp for any
 * map of this shape: the operand sized for all B*B bins (for
 * GSP_PREC_STRUCTURED tens of MB instead of the tensor). */
size_t gsp_cp_workspace_bytes(int N, int levels, int bins, int rank, int precision);

/* The same for a map in which `occupied_bins` of the B*B bins occur (as
 * counted by gsp_cp_count_bins): the operand and every array sized by its
 * columns hold only the columns gsp_cp_prepare keeps (see there), e.g. 2.5 GB
 * instead of 23 GB for the BF16 operand of a 1024^2 map with 11 levels, 32x32
 * bins of which 67 occur, rank 64.  0 for invalid arguments
 * (occupied_bins outside 1 .. B*B).  gsp_cp_prepare returns
 * GSP_ERR_WORKSPACE, having enqueued only the bin count, when the map it is
 * given needs more. */
size_t gsp_cp_workspace_bytes_for_bins(int N, int levels, int bins, int rank, int precision,
                                       int occupied_bins);

/* Count the bins that occur in the normal map (d_normal_xy, binned as in
 * gsp_bin_normals) or in the level-0 slice of d_hist, the count that sizes a
 * workspace by gsp_cp_workspace_bytes_for_bins.  B*B when B*B < 256 (the
 * operand then keeps every bin).  d_ws: gsp_cp_count_bins_workspace_bytes()
 * bytes of scratch (the first bytes of any CP workspace of this N and B
 * will do).  Synchronises `stream` to write *h_occupied (host). */
size_t gsp_cp_count_bins_workspace_bytes(int N, int bins);
int gsp_cp_count_bins(const int32_t* d_hist, const float* d_normal_xy, int N, int levels,
                      int bins, void* d_ws, size_t ws_bytes, int32_t* h_occupied,
                      uint32_t* d_status, gsp_stream stream);

/* Byte offset in a CP workspace of the operand gsp_cp_prepare builds
 * (dense-path precisions; 0 for GSP_PREC_STRUCTURED, which builds none).
 * The workspace starts with a head of fixed size (bin map, column tables,
 * the FP64 ALS arrays), then the operand. */
size_t gsp_cp_operand_offset(int N, int levels, int bins, int rank, int precision);

/* Build the MTTKRP operand (the NDF tensor in the precision's input type,
 * [l][y][x][c]: BF16 for GSP_PREC_BF16 / _BF16_1X, else FP32, on the TF32
 * grid for GSP_PREC_TF32; it occupies levels*N*N*C elements from byte
 * gsp_cp_operand_offset() of d_ws) and ||T||^2 inside the workspace.  The operand keeps only the bins
 * that occur somewhere in the map (all other bins are zero in every
 * footprint): column c < n holds the c-th occurring bin (s*B + t, in
 * increasing order), columns n .. C-1 are zero, C = n rounded up to a multiple
 * of 16 for the tensor-core precisions and of 128 for GSP_PREC_FP32 (at most
 * B*B); with B*B < 256, C = B*B and column c is bin c.  The
 * call synchronises `stream` once to learn C (gsp_cp_operand_cols reports
 * it).  Dropping the all-zero columns changes only the order of the FP32
 * accumulation against the full B*B operand.  Exactly one of d_hist
 * (int32 histograms from gsp_build_footprint_ndfs) and d_normal_xy (the normal
 * map: the histograms are then produced level by level straight into the
 * operand, never stored as int32) must be non-NULL; with d_hist the occurring
 * bins are those of its level-0 slice (one count of 1 per texel, checked as
 * for GSP_PREC_STRUCTURED below).  GSP_PREC_STRUCTURED builds
 * no operand: it keeps the bin map (binned from d_normal_xy, or read from the
 * level-0 slice of d_hist, which holds a single count of 1 per texel; a slice
 * that does not sets GSP_DEV_BAD_QUERY in d_status and that texel's bin to 0)
 * and ||T||^2 (from the histogram counts' sums of squares). */
int gsp_cp_prepare(const int32_t* d_hist, const float* d_normal_xy, int N, int levels,
                   int bins, int rank, const gsp_als_opts* opts, void* d_ws,
                   size_t ws_bytes, uint32_t* d_status, gsp_stream stream);

/* The operand columns of a workspace prepared by gsp_cp_prepare (dense-path
 * precisions): h_cols[0] = bins occurring in the map, h_cols[1] = columns C
 * per footprint.  Synchronises `stream`. */
int gsp_cp_operand_cols(int N, int levels, int bins, int rank, int precision, const void* d_ws,
                        size_t ws_bytes, int32_t* h_cols, gsp_stream stream);

/* Run ALS sweeps on the operand prepared in d_ws.  `f` holds the starting
 * factors on entry (e.g. seeded U[0,1)) and the result on exit.  Mode order
 * per sweep: x, y, l, s, t; each update is the exact least-squares solution
 * A_n = M_n V^-1 with V the Hadamard product of the other modes' FP64 Gram
 * matrices (Cholesky; pseudo-inverse fallback), then 2-norm column
 * normalisation into lambda.  V does not depend on the mode's MTTKRP, so its
 * factorisation and inverse run on a side stream the call creates, concurrently
 * with that MTTKRP; the side stream starts after the work already queued on
 * `stream`, and everything the call queues joins back into `stream`.  While
 * `stream` is being captured into a CUDA graph everything stays on `stream`
 * (capture then needs h_report == NULL, tol == 0 and a workspace prepared in
 * this process, whose operand column count the library then knows without
 * reading the device). */
int gsp_cp_sweeps(int N, int levels, int bins, int rank, const gsp_als_opts* opts,
                  const gsp_cp_factors* f, gsp_als_report* h_report, void* d_ws,
                  size_t ws_bytes, gsp_stream stream);

/* gsp_cp_prepare followed by gsp_cp_sweeps. */
int gsp_cp_decompose(const int32_t* d_hist, const float* d_normal_xy, int N, int levels,
                     int bins, int rank, const gsp_als_opts* opts, const gsp_cp_factors* f,
                     gsp_als_report* h_report, void* d_ws, size_t ws_bytes,
                     uint32_t* d_status, gsp_stream stream);

/* The five MTTKRPs of the prepared operand for fixed factors f (lambda unused):
 * M_n[i][r] = sum over the other four indices of T * prod_{m != n} f_m[i_m][r].
 * d_m[0..4] = M_x [N][R], M_y [N][R], M_l [levels][R], M_s [B][R], M_t [B][R]
 * (FP32, written).  Used to check the contraction kernels one by one. */
int gsp_cp_mttkrp(int N, int levels, int bins, int rank, int precision,
                  const gsp_cp_factors* f, float* const d_m[5], void* d_ws,
                  size_t ws_bytes, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* a5/a6 -- query tables and batched range query (Sec. 4.3-4.4, Eq. 4-5)     */
/* ------------------------------------------------------------------------ */

/* One CP-compressed material.  Factor pointers are read by the query kernels;
 * `tables` (gsp_query_table_floats() floats, caller-owned, 16-byte aligned) is
 * written by gsp_build_query_tables and holds, in order:
 *   flw  [levels][R]       fl * lambda (the CP weights folded into the level factor),
 *                          padded to a multiple of 4 floats
 *   sats [B+1][3][R]       1D summed-area table of fs, row i = three planes of R
 *                          floats: hi, lo and fs[i] (0 at i = B), with
 *                          hi + lo = sum_{k<i} fs[k] (FP64 sum split into two
 *                          FP32); a range's partial end bins are weighted from the
 *                          bin values, the whole bins between them from hi + lo
 *   satt [B+1][3][R]       the same for ft.
 * The query kernels read consecutive ranks of a plane as vector loads when
 * every rank is a multiple of 32 and fx, fy are 16-byte aligned.              */
typedef struct gsp_material {
  int32_t N, levels, bins, rank;
  const float* fx;
  const float* fy;
  const float* fl;
  const float* fs;
  const float* ft;
  const float* lambda;
  float* tables;
} gsp_material;

/* 32-byte query descriptor (arrays of them must be 16-byte aligned).  x, y: texel, taken mod N.  level: footprint level,
 * clamped to [0, levels-1], blended linearly between floor(level) and the next
 * level.  [s0, s1] x [t0, t1]: angular range in bin units (bin k = [k, k+1)),
 * clamped to [0, B] and reordered if reversed; a zero-width side is a point
 * query of the bin holding it.  material: index into the materials array. */
typedef struct gsp_query {
  int32_t x, y;
  float level, s0, s1, t0, t1;
  uint32_t material;
} gsp_query;

size_t gsp_query_table_floats(int levels, int bins, int rank);

/* Fill h_mat->tables from its factors (1D SAT per angular factor, Sec. 4.4). */
int gsp_build_query_tables(const gsp_material* h_mat, gsp_stream stream);

/* Launch shape of the range-query kernel.  NULL, or a field of 0, takes the
 * library's default: 8 lanes per query when some rank is >= 64, else 4; 8
 * CTAs per SM; 256 threads; 4 queries per grab.  Results do not depend on it. */
typedef struct gsp_query_tuning {
  int32_t lanes_per_query; /* 4, 8, 16 or 32 */
  int32_t blocks_per_sm;   /* persistent CTAs per SM (1 .. 32)   */
  int32_t threads;         /* threads per CTA (32 .. 256, multiple of 32) */
  int32_t chunk;           /* batches of 32 queries a warp claims per grab (1 .. 64) */
} gsp_query_tuning;

/* Batched range queries (Eq. 5 extended to five modes):
 *   q = sum_r fx[x,r] fy[y,r] ((1-f) flw[l0,r] + f flw[l1,r]) Sbar_r Tbar_r,
 *   Sbar_r = (F_r(s1) - F_r(s0)) / (s1 - s0),  F_r(s) = P_r[floor s] + frac(s) fs[floor s, r],
 * two summed-area-table look-ups per range end (Sec. 4.4).  h_mats: host array
 * of n_mats (<= GSP_MAX_MATERIALS) materials with built tables.  d_q: n queries;
 * d_out: n floats, written.  A malformed query writes NaN and sets
 * GSP_DEV_BAD_QUERY.  d_ws: 16 bytes of scratch (work counter) or more.
 * Capturable in a CUDA graph (no allocation, no synchronisation). */
int gsp_range_query(const gsp_material* h_mats, int n_mats, const gsp_query* d_q, int64_t n,
                    float* d_out, uint32_t* d_status, const gsp_query_tuning* tuning,
                    void* d_ws, size_t ws_bytes, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* f1 -- hierarchical NDF importance sampling from range queries (Sec. 5.2)  */
/* ------------------------------------------------------------------------ */

/* A footprint to sample: texel (x, y) taken mod N, level clamped to
 * [0, levels-1] and blended between floor(level) and floor(level) + 1 as in
 * gsp_query, material: index into the materials array.  16 bytes. */
typedef struct gsp_sample_query {
  int32_t x, y;
  float level;
  uint32_t material;
} gsp_sample_query;

/* Uniform random numbers in [0, 1) each sample consumes: u[k] chooses the
 * quad at subdivision step k (k < log2 B <= 6), u[6] and u[7] place the sample
 * inside the final bin. */
#define GSP_SAMPLE_UNIFORMS 8

/* Hierarchical importance sampling of the NDF image of each footprint (Sec.
 * 5.2, Fig. sampling): start from the whole B x B image; split the current
 * square into four quads at its midpoints, take their average NDF values by
 * four range queries (Sec. 4.3), clamp negative averages (possible for a CP
 * approximation) to 0 and choose one quad with probability proportional to
 * its average (quads in the order (s low, t low), (s low, t high), (s high, t
 * low), (s high, t high): the first k with u * total < cumulative sum); if all
 * four are 0 the choice is uniform.  After log2 B steps the square is one bin;
 * the sample is placed uniformly inside it.  Output per sample, d_out [n][4]:
 *   s, t        the sampled direction in bin units, in [0, B)
 *   pmf         probability of the chosen bin (product of the step probabilities;
 *               for a non-negative tensor the bin's value / the image sum)
 *   value       the range average of the chosen bin, i.e. its NDF value.
 * Requires every material's bin count to be a power of two <= 64
 * (GSP_ERR_UNSUPPORTED otherwise) and built tables.  d_u: [n][GSP_SAMPLE_UNIFORMS]
 * floats.  A malformed sample (bad material or non-finite level) writes NaN
 * and sets GSP_DEV_BAD_QUERY.  Capturable in a CUDA graph. */
int gsp_sample_ndf(const gsp_material* h_mats, int n_mats, const gsp_sample_query* d_q,
                   int64_t n, const float* d_u, float* d_out, uint32_t* d_status,
                   gsp_stream stream);

/* A range query at a fractional texel position: x, y in texel units (|x|,
 * |y| < 2^30), the other fields as in gsp_query.  32 bytes. */
typedef struct gsp_query_f {
  float x, y;
  float level, s0, s1, t0, t1;
  uint32_t material;
} gsp_query_f;

/* gsp_range_query at fractional positions (Sec. 4.1: the NDF of an arbitrary
 * footprint by interpolation between neighbouring footprint samples): the
 * bilinear blend over the texels floor(x) + {0, 1}, floor(y) + {0, 1} (mod N)
 * of their range queries, computed as one query with the fx and fy rows
 * interpolated (the CP tensor is multilinear).  At integer positions the
 * result equals gsp_range_query's.  A non-finite or too large x or y counts
 * as a malformed query. */
int gsp_range_query_interp(const gsp_material* h_mats, int n_mats, const gsp_query_f* d_q,
                           int64_t n, float* d_out, uint32_t* d_status,
                           const gsp_query_tuning* tuning, void* d_ws, size_t ws_bytes,
                           gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* f4 -- environment-lighting prefiltering queries (Sec. 5.4)                */
/* ------------------------------------------------------------------------ */

/* A spherical Gaussian lobe of the environment light (Sec. 5.4):
 * G(v) = amplitude * exp(sharpness * (dot(v, axis) - 1)), axis a unit vector. */
typedef struct gsp_sg {
  float axis[3];
  float amplitude;
  float sharpness;
  float pad[3];
} gsp_sg; /* 32 bytes */

/* One shading record: footprint (x, y, level, material as in gsp_query), the
 * unit outgoing direction wo, and the index of the SG lobe the light sampling
 * chose.  32 bytes. */
typedef struct gsp_env_record {
  int32_t x, y;
  float level;
  float wo[3];
  uint32_t sg;
  uint32_t material;
} gsp_env_record;

/* Range-query descriptors for environment-light prefiltering (Sec. 5.4), one
 * per record, written to d_q (then answered by gsp_range_query):
 *   theta = arccos((ln eps - ln A) / lambda + 1)       (compact-eps support of the lobe;
 *           theta = pi when the argument is below -1, theta = 0 when A <= eps)
 *   Q     = B * theta / pi                             (side of the square in bins; the
 *                                                      paper's 256-pixel images -> B bins)
 *   h     = normalize(wo + axis), centre (s, t) = ((h.x + 1) B / 2, (h.y + 1) B / 2)
 *   range [s - Q/2, s + Q/2] x [t - Q/2, t + Q/2]   (clamped by the query itself).
 * B is the bin count of the record's material (h_mats as for gsp_range_query).
 * A record whose SG index or material is out of range, or with wo = -axis,
 * gets level = NaN (the query then reports GSP_DEV_BAD_QUERY). */
int gsp_env_queries(const gsp_material* h_mats, int n_mats, const gsp_sg* d_sgs, int n_sgs,
                    const gsp_env_record* d_rec, int64_t n, float eps, gsp_query* d_q,
                    gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* f2 -- the clustered compression layout of Sec. 4.2                        */
/* ------------------------------------------------------------------------ */
/* Sec. 4.2 compresses groups of angular blocks instead of one global tensor.
 * Every footprint histogram (B x B bins, from gsp_build_footprint_ndfs) is
 * split into t x t blocks, t = 16 (bins a multiple of 16, B >= 16).  The
 * blocks at one block position (bs, bt) of the footprints centred in one
 * 8 x 8-texel region (cx, cy) (N >= 8) form group
 *   j = ((cy * (N / 8) + cx) * nb + bs) * nb + bt,   nb = bins / 16.
 * A group keeps its non-blank blocks (some count > 0) in the order level, then
 * y, then x; z numbers them; completely blank blocks are dropped.  Group j's
 * tensor D_j[s'][t'][z] = c_l * H_l[y][x][16 bs + s'][16 bt + t'] (c_l the
 * density scale B^2/(4*4^l), or 1 with raw counts) is decomposed by its own
 * CP-ALS: D_j ~ sum_r lambda_r X_r o Y_r o Z_r (Eq. 3), modes X (s'), Y (t'),
 * Z (z), in that order per sweep. */

/* Number of groups (N / 8)^2 * (bins / 16)^2 (0 if the shape is unsupported)
 * and the scratch bytes gsp_cluster_layout needs. */
int gsp_cluster_groups(int N, int levels, int bins);
size_t gsp_cluster_layout_bytes(int N, int levels, int bins);

/* Build the layout from int32 histograms d_hist [levels][N][N][B][B].
 *  d_offsets [groups + 1]: group j's members are rows offsets[j] ..
 *            offsets[j + 1] - 1 (written);
 *  d_members [levels * N * N * nb * nb] capacity: packed member (level << 20 |
 *            y << 10 | x) of every row (written);
 *  d_zmap    [levels][N][N][nb * nb]: z of the footprint's block in its group,
 *            -1 if blank (written);
 *  h_stats   [2] host: total members, largest group (the call synchronises).
 * Deterministic; bit-exact. */
int gsp_cluster_layout(const int32_t* d_hist, int N, int levels, int bins, int32_t* d_offsets,
                       int32_t* d_members, int32_t* d_zmap, int64_t* h_stats, void* d_ws,
                       size_t ws_bytes, gsp_stream stream);

/* Shared memory per group CTA of gsp_cluster_als (0 if unsupported); the call
 * needs at most 227 KB. */
size_t gsp_cluster_als_smem(int rank, int max_members);

/* Batched CP-ALS of every group, one CTA per group (rank 8, 16 or 32).
 *  d_X, d_Y [groups][16][rank], d_Z [total members][rank]: initial factors
 *  in, result out (unit 2-norm columns); d_lambda [groups][rank] out.
 *  Every group runs until |fit_k - fit_(k-1)| < tol (Sec. 4.2: 1e-4; 0: never)
 *  or max_sweeps; d_sweeps [groups] (int32) and d_fit [groups] (FP64, 1 -
 *  ||D - D_hat|| / ||D||) receive what each group did; empty groups report 0.
 *  FP32 MTTKRP products with compensated sums, FP64 Gram / Cholesky / inverse /
 *  apply / normalisation; a Gram system that is not positive definite is
 *  retried with a growing ridge and flags GSP_DEV_NUMERIC in d_status.
 *  d_ws: at least levels * 8 bytes. */
int gsp_cluster_als(const int32_t* d_hist, int N, int levels, int bins, int rank,
                    const int32_t* d_offsets, const int32_t* d_members, int max_members,
                    float* d_X, float* d_Y, float* d_Z, float* d_lambda, int max_sweeps,
                    double tol, int raw_counts, int32_t* d_sweeps, double* d_fit,
                    uint32_t* d_status, void* d_ws, size_t ws_bytes, gsp_stream stream);

/* Query tables of the decomposed groups (Sec. 4.4): d_xsat, d_ysat
 * [groups][17][rank][4] floats {hi, lo, f[i], f[i-1]} with hi + lo =
 * sum_{k < i} f[k] (FP64 sums split into two FP32); d_zw [total members][rank]
 * = lambda * Z. */
int gsp_cluster_tables(int N, int levels, int bins, int rank, const int32_t* d_offsets,
                       const float* d_X, const float* d_Y, const float* d_Z,
                       const float* d_lambda, float* d_xsat, float* d_ysat, float* d_zw,
                       gsp_stream stream);

/* Range query against the clustered layout: gsp_query descriptors (material
 * ignored), semantics of gsp_range_query (x, y wrap; level clamped and blended
 * linearly; bin ends clamped to [0, B] and ordered; zero width = the point
 * value of the bin holding the end).  A range that crosses block borders is
 * split at them (Sec. 4.4) and the parts weighted by their share of the
 * range; a blank block reads 0.  d_out [n] FP32; malformed -> NaN and
 * GSP_DEV_BAD_QUERY. */
int gsp_cluster_range_query(int N, int levels, int bins, int rank, const int32_t* d_offsets,
                            const int32_t* d_zmap, const float* d_xsat, const float* d_ysat,
                            const float* d_zw, const gsp_query* d_q, int64_t n, float* d_out,
                            uint32_t* d_status, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* a7 -- adjoint of the range query and the refinement step                  */
/* ------------------------------------------------------------------------ */

/* Gradient buffers of one material, FP32, same shapes as the factors; the
 * level gradient is with respect to flw = fl * lambda. */
typedef struct gsp_material_grad {
  float* dfx;
  float* dfy;
  float* dflw;
  float* dfs;
  float* dft;
} gsp_material_grad;

/* Scratch of gsp_range_query_backward for these materials: the gradients of
 * each material's summed-area-table prefix sums (2 (bins + 1) rank floats),
 * then 128 private copies of every material's small gradient tables ((levels
 * + 2 (bins + 1)) rank floats each), which the adjoint's CTAs accumulate into
 * (a copy is shared by at most two CTAs) and one kernel sums afterwards.
 * 0 when h_mats is NULL or n_mats is outside 1 .. GSP_MAX_MATERIALS.  The
 * materials' own fields are not checked here (levels, bins and rank are read
 * as given).  gsp_range_query_backward rejects a malformed material before it
 * uses the workspace: with GSP_ERR_INVALID_ARG, or with GSP_ERR_WORKSPACE when
 * ws_bytes is below the size computed from that material (the size test comes
 * first). */
size_t gsp_backward_workspace_bytes(const gsp_material* h_mats, int n_mats);

/* Accumulate (+=) d(sum_i g_i q_i)/d(factors) into h_grads[m] for every
 * material m; d_gout holds the n upstream gradients g_i.  The angular
 * gradients go first to the summed-area-table entries the query read and are
 * turned into factor gradients by one suffix sum per material. */
int gsp_range_query_backward(const gsp_material* h_mats, int n_mats, const gsp_query* d_q,
                             int64_t n, const float* d_gout, const gsp_material_grad* h_grads,
                             void* d_ws, size_t ws_bytes, uint32_t* d_status,
                             gsp_stream stream);

/* gsp_range_query_backward without a caller workspace, for callers that cannot
 * allocate device memory: a shading or sampling plugin that only receives the
 * device pointers its host application hands it and has no allocator of its
 * own, or a frame loop that must not call cudaMalloc because it synchronises
 * the whole device.  The paper has no counterpart; this is a calling
 * convention of this library.
 *  The scratch (gsp_backward_workspace_bytes() of it: the per-material
 *  gradients of the summed-area-table prefix sums and the private copies of
 *  the small gradient tables) comes from one fixed array of
 *  GSP_BACKWARD_NOALLOC_MAX_BYTES in device memory that the library defines;
 *  every GPU that loads the library holds it until the process exits.  Larger
 *  material sets are rejected with GSP_ERR_WORKSPACE before anything is
 *  enqueued, and malformed materials with GSP_ERR_INVALID_ARG.  The call
 *  allocates nothing and calls no allocating routine.
 *  The first call on a device looks up the array's device address with that
 *  device current (no work is enqueued by that step).  If no kernel of the
 *  library has run on that device yet, that lookup is what loads the
 *  library's device code there (CUDA loads modules lazily): the loader then
 *  places the module's own globals, this array among them, in device memory
 *  and may synchronise the device.  So make the first call at initialisation,
 *  before any stream capture and before the frame loop that must not stall.
 *  The address is kept per device for the life of the process: after a
 *  cudaDeviceReset() in the calling process it is stale, and this call must
 *  not be used on that device again.  All calls share the one array and it keeps the
 *  last call's contents: each call clears the part it uses on `stream` before
 *  its kernels run, so calls must not overlap on the GPU (two streams running
 *  this call at the same time race on the array).  Arguments and results are
 *  those of gsp_range_query_backward. */
#define GSP_BACKWARD_NOALLOC_MAX_BYTES (4u << 20)
int gsp_range_query_backward_noalloc(const gsp_material* h_mats, int n_mats,
                                     const gsp_query* d_q, int64_t n, const float* d_gout,
                                     const gsp_material_grad* h_grads, uint32_t* d_status,
                                     gsp_stream stream);

/* One Adam step (Kingma & Ba 2015) on n FP32 parameters in place:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps). */
int gsp_adam_step(float* d_param, const float* d_grad, float* d_m, float* d_v, int64_t n,
                  int step, float lr, float beta1, float beta2, float eps, gsp_stream stream);

/* ------------------------------------------------------------------------ */
/* misc                                                                      */
/* ------------------------------------------------------------------------ */

/* Kernel timing for measurement.  When enabled, the library records a pair of
 * CUDA events on the launching stream around every launch of the kernels
 * below (id = index).  gsp_profile_read synchronises those events and returns
 * the launch count and summed device time since the last reset.  Off by
 * default; keep it off while capturing CUDA graphs.
 *   0 bins, 1 (unused), 2 box_hist, 3 cast, 4 mttkrp_xy, 5 mttkrp_lst,
 *   6 als_small, 7 tables, 8 range_query, 9 range_query_backward, 10 adam,
 *   11 struct_tables, 12 struct_side, 13 struct_bins (GSP_PREC_STRUCTURED),
 *   14 solve (Cholesky and inverse of the ALS Gram system, on the side stream
 *   gsp_cp_sweeps runs it on, concurrently with the mode's MTTKRP) */
#define GSP_PROFILE_SLOTS 15
int gsp_profile_enable(int on);
void gsp_profile_reset(void);
int gsp_profile_read(int id, int64_t* h_launches, double* h_total_ms);
const char* gsp_profile_name(int id);
/* Kernel launches issued by this library since the process started. */
uint64_t gsp_kernel_launches(void);

/* Failure-path self-test of the bounded device waits (no fault, no hang).
 * Launches one CTA that waits on an mbarrier nothing ever arrives at, through
 * the same bounded wait the tensor-core kernels use for their TMA / MMA
 * pipelines.  The wait gives up after its clock budget (4e9 SM cycles, about
 * 2 s at GB300 clocks), the CTA ORs GSP_DEV_TIMEOUT into *d_err (device
 * word, required) and returns, leaving the context usable.  Returns GSP_OK
 * once launched; the status bit arrives asynchronously on `stream`. */
int gsp_selftest_wait_timeout(uint32_t* d_err, gsp_stream stream);

/* Self-test of the FP64 reciprocal on the Cholesky pivot chain of the CP-ALS
 * solve (Newton-Raphson from the FP32 reciprocal): d_out[i] = that reciprocal
 * of d_in[i], FP64 device arrays of n elements (n >= 0), so that it can be
 * checked against the correctly rounded 1/d. */
int gsp_selftest_recip(const double* d_in, int64_t n, double* d_out, gsp_stream stream);

const char* gsp_strerror(int status);
/* cudaError_t value of the last failing CUDA call in this thread (0 if none). */
int gsp_last_cuda_error(void);
/* Library version, major * 10000 + minor * 100 + patch.  2.0.0: query tables
 * as hi / lo / value planes (gsp_query_table_floats changed) and the compacted
 * CP-ALS operand (gsp_cp_operand_cols). */
int gsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSP_H */
