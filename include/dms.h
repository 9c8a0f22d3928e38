/*
 * dms.h -- C ABI of the GB300-native Discrete Morse Sandwich hot path.
 *
 * The method is the one of "Distributed Discrete Morse Sandwich" (arXiv
 * 2505.21266): a scalar field on a 3D regular grid, triangulated by the
 * Freudenthal (Kuhn) split, goes through
 *   (i)   the global vertex order            (Sec. 2.1, Sec. 3 "Array Preconditioning"),
 *   (ii)  Robins et al.'s lower-star discrete gradient (Sec. 2.3),
 *   (iii) critical-simplex extraction         (Sec. 2.5 "zero-persistence skip", Sec. 3),
 *   (iv)  the extremum-saddle pairs D0 and D2 (Sec. 2.5, Alg. 1 and its dual; Sec. 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Vertex v = x + nx*(y + ny*z), x fastest (Sec. 2.1, "vertex offsets in
 *    memory").  Each dim must be >= 2 and nx*ny*nz < 2^32 - 1.
 *  - Simplices are chains of cube corners (Kuhn split along the (1,1,1)
 *    diagonal), anchored at their componentwise-smallest vertex a.  A cube
 *    corner is a 3-bit mask (bit0 = +x, bit1 = +y, bit2 = +z).  Ids (int64):
 *      vertex   v
 *      edge     7a + k,  k -> corner {1,2,4,3,5,6,7}[k]          ({a, a+c})
 *      triangle 12a + k, k -> (p,q) {(1,3),(2,3),(1,5),(4,5),(2,6),(4,6),
 *                                   (1,7),(2,7),(4,7),(3,7),(5,7),(6,7)}[k]
 *                                                              ({a, a+p, a+q})
 *      tet      6a + k,  k -> (c1,c2) {(1,3),(1,5),(2,3),(2,6),(4,5),(4,6)}[k]
 *                                                    ({a, a+c1, a+c2, a+7})
 *    An id names a simplex only if all of its vertices are in the grid.
 *  - Simplices are compared by the orders of their vertices listed by
 *    decreasing value, lexicographically, a proper prefix first (Sec. 2.1).
 *  - Every pointer argument is a DEVICE pointer owned by the caller unless
 *    marked "host".  No entry point allocates memory.  Work is enqueued on
 *    `stream` and is asynchronous unless stated otherwise.
 *  - Return value: a dms_status for errors the host can see (NULL pointers,
 *    bad dims, short workspace or capacity known on the host, CUDA launch
 *    errors).  Errors that depend on the data (NaN input, capacity exceeded,
 *    an iteration limit reached) are OR-ed as (1 << status) into the device
 *    word *dstatus, which the caller zeroes beforehand and reads after a
 *    synchronisation.
 */
#ifndef DMS_H_
#define DMS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dms_dims {
  int32_t nx, ny, nz; /* x fastest */
} dms_dims;

/* One persistence pair (Sec. 2.4): the pair is embedded at
 * (f(birth simplex), f(death simplex)), f(s) being the highest vertex value
 * of s; birth_vtx / death_vtx are those highest vertices.  D0: birth_id is a
 * minimum (vertex id), death_id an edge id.  D2: birth_id is a triangle id,
 * death_id a tetrahedron id.  The essential D0 class has death_id = -1,
 * death = +inf, death_vtx = 0. */
typedef struct dms_pair {
  int64_t birth_id;
  int64_t death_id;
  float birth;
  float death;
  uint32_t birth_vtx;
  uint32_t death_vtx;
} dms_pair;

/* A field of a batch: its vertices occupy [offset, offset + nx*ny*nz) of the
 * concatenated per-vertex arrays (fields adjacent, offsets increasing from 0). */
typedef struct dms_field_desc {
  int64_t offset;
  int32_t nx, ny, nz; /* each >= 2, x fastest */
  int32_t reserved;   /* 0 */
} dms_field_desc;

typedef enum dms_status {
  DMS_OK = 0,
  DMS_ERR_NULL = 1,       /* a required pointer is NULL */
  DMS_ERR_DIMS = 2,       /* a dim < 2, or nx*ny*nz >= 2^32 - 1 */
  DMS_ERR_NAN = 3,        /* the field holds a NaN (device-detected) */
  DMS_ERR_CAPACITY = 4,   /* an output list is too short; counts hold the need */
  DMS_ERR_WORKSPACE = 5,  /* ws_bytes smaller than the *_workspace_size query */
  DMS_ERR_CUDA = 6,       /* a CUDA call failed */
  DMS_ERR_TIMEOUT = 7,    /* an iterative stage hit its iteration limit */
  DMS_ERR_ARG = 8,        /* another invalid argument */
  DMS_ERR_TOO_LARGE = 9   /* the grid exceeds the fixed scratch of a no-alloc entry point */
} dms_status;

/* Human-readable text for a dms_status (static storage). */
const char* dms_status_string(int status);

/* Instrumentation, not part of the method: the number of CUDA kernels this
 * library has launched since it was loaded (every entry point adds its own
 * launches).  Not thread-safe; the benchmark reads it around its timed
 * region. */
int64_t dms_launch_count(void);

/* Number of vertices of the grid, or 0 if the dims are invalid. */
int64_t dms_num_vertices(dms_dims d);

/* ------------------------------------------------------------------ (i) ---
 * dms_order -- the global vertex order (Sec. 2.1; Sec. 3 "Array
 * Preconditioning"): order[v] = position of v in the stable sort of the
 * vertices by increasing f, -0.0 equal to +0.0, ties broken by the vertex
 * offset v.  ±inf are ordinary values; a NaN anywhere sets (1 << DMS_ERR_NAN)
 * in *dstatus (order is then unspecified).
 *   f       [n] float32, read only.
 *   order   [n] uint32 out (a permutation of 0..n-1).
 *   ws      workspace of at least dms_order_workspace_size(d) bytes,
 *           256-byte aligned, contents need not be initialised.
 *   dstatus one int32 the caller zeroed.
 */
size_t dms_order_workspace_size(dms_dims d);
int dms_order(const float* f, dms_dims d, uint32_t* order, void* ws, size_t ws_bytes,
              int32_t* dstatus, void* stream);

/* ----------------------------------------------------------------- (ii) ---
 * dms_gradient -- Robins et al.'s discrete gradient, computed vertex by vertex
 * on its lower star (Sec. 2.3): ProcessLowerStars with priority queues on
 * the lexicographic key, the steepest lower edge paired with the vertex.
 *   order   [n] uint32 from dms_order (any permutation works: it IS the order).
 *   desc    [n] uint8 out.  desc[v] = 0..13: v is paired with its edge to the
 *           neighbour v + off[desc] where off[s] is +c for s < 7 and -c for
 *           s >= 7, c = corner {1,2,4,3,5,6,7}[s % 7]; 15: v is critical (a
 *           minimum).
 *   rec     [n] uint64 out, one record per anchor a, describing the 7 edges,
 *           12 triangles and 6 tetrahedra anchored at a:
 *             bits 3k..3k+2 (edge k):  0 = absent or paired with its top
 *                vertex, 1..6 = paired with the (code-1)-th triangle holding
 *                it, cofacets listed by increasing id on the unbounded
 *                lattice, 7 = critical;
 *             bit 21+k (triangle k): 1 = critical;
 *             bits 33+3k..35+3k (tet k): 0 = absent, 1..4 = paired with the
 *                facet that omits vertex (code-1) of the chain
 *                a < a+c1 < a+c2 < a+7, 7 = critical;
 *             other bits 0.
 *           Triangles paired with an edge are recorded at that edge, those
 *           paired with a tetrahedron at the tetrahedron.
 *   crit_counts [4] int64 out: number of critical simplices per dimension
 *           (overwritten, not accumulated).  crit_counts[0] < 0 after the
 *           call means that a TMA copy of the order field into shared memory
 *           did not complete within the kernel's wait limit: the outputs are
 *           then invalid (read it as DMS_ERR_TIMEOUT).
 * When nx is a multiple of 4 and order is 16-byte aligned, the kernel stages
 * the order field through TMA (cp.async.bulk.tensor tile loads of one slab
 * window each, two slabs ahead); otherwise through ordinary loads.  The
 * results are the same.  The launch tiles y by 24 rows in the grid's second
 * dimension, so ny is at most 24 * 65535 = 1,572,840; a taller grid fails
 * to launch and returns DMS_ERR_CUDA (the batch call has no such limit).
 */
int dms_gradient(const uint32_t* order, dms_dims d, uint8_t* desc, uint64_t* rec,
                 int64_t* crit_counts, void* stream);

/* ---------------------------------------------------------------- (iii) ---
 * dms_critical -- stream compaction of the critical simplices ("zero-
 * persistence skip", Sec. 2.5; "Extract & sort", Sec. 3): crit_k receives the
 * ids of the critical k-simplices in increasing id order.
 *   desc, rec  from dms_gradient.
 *   crit0..3   int64 out arrays of capacity cap[k] (host array of 4).
 *   counts     [4] int64 out: the number of critical k-simplices.  If one
 *              exceeds cap[k], (1 << DMS_ERR_CAPACITY) is set in *dstatus and
 *              only the first cap[k] ids are written.
 *   ws         at least dms_critical_workspace_size(d) bytes.
 */
size_t dms_critical_workspace_size(dms_dims d);
int dms_critical(const uint8_t* desc, const uint64_t* rec, dms_dims d, int64_t* crit0,
                 int64_t* crit1, int64_t* crit2, int64_t* crit3, const int64_t* cap,
                 int64_t* counts, void* ws, size_t ws_bytes, int32_t* dstatus, void* stream);

/* dms_critical_noalloc -- the same compaction as dms_critical, for callers
 * that cannot allocate device memory (no workspace argument).  The paper has
 * no counterpart; this is a deployment variant.
 *
 * Callers that run inside an allocator-free region of another framework,
 * plug-ins given only their input and output buffers, or real-time loops
 * that must not call cudaMalloc (it may synchronise the device) pass the
 * same inputs and outputs as to dms_critical; the scratch (about 8 MiB) is a
 * static array in the library image, present on every GPU that loads the
 * library until the process exits.  Grids of more than
 * dms_critical_noalloc_max_vertices() = 2^30 vertices return
 * DMS_ERR_TOO_LARGE.  The first call on a device looks up that device's
 * address of the array (cudaGetSymbolAddress), so make a first call on each
 * device before capturing streams.  The looked-up address stays cached for
 * the life of the process: after a cudaDeviceReset (or any other teardown of
 * the device's primary context) the cached address is stale, so do not call
 * this entry point on a device after resetting it.  Every call shares the array: calls whose
 * GPU work may overlap (other streams, other host threads) race on it.  The
 * array needs no clearing: each call writes all the scratch it reads.
 * Nothing is allocated (no cudaMalloc, cudaFree or allocating library call).
 */
int64_t dms_critical_noalloc_max_vertices(void);
int dms_critical_noalloc(const uint8_t* desc, const uint64_t* rec, dms_dims d, int64_t* crit0,
                         int64_t* crit1, int64_t* crit2, int64_t* crit3, const int64_t* cap,
                         int64_t* counts, int32_t* dstatus, void* stream);

/* ----------------------------------------------------------------- (iv) ---
 * dms_diagram_d0d2 -- the extremum-saddle persistence pairs (Sec. 2.5, Alg. 1,
 * Sec. 4.1-4.2).  D0: from both vertices of every critical edge the
 * descending v-path is followed to a minimum; the triplets (edge, t0, t1)
 * with t0 != t1 are taken in increasing edge order and, with a union-find
 * over minima, the younger (higher) root dies against the edge.  D2: from the
 * two cofacets of every critical triangle the dual (ascending) v-path is
 * followed to a critical tetrahedron, or to a virtual OUTSIDE node when the
 * path leaves the grid; triangles are taken in decreasing order and the lower
 * maximum dies (OUTSIDE never dies).  Alg. 1 pairs nothing at a saddle whose
 * ends lighter saddles already join, so only the saddles of the minimum
 * spanning forest of the extremum graph matter: Boruvka rounds find them
 * first (every component joins across its lightest live saddle).  The
 * pairing then runs in rounds over those saddles that are exact: a round
 * merges every saddle that is the lightest live saddle of both of its
 * components, or the lightest of a component whose other side is older;
 * both choices are the ones Alg. 1 makes at that saddle's turn.
 * Paths that meet share their tail: a walk that reaches a vertex (D0) or a
 * tetrahedron (D2) another walk has passed stops and takes that walk's end.
 *   f, order, desc, rec   as above;  crit0..3 and n_crit (HOST array of 4)
 *                         from dms_critical; n_crit[1], n_crit[2] < 2^30.
 *   d0   [cap0] out: D0 pairs in increasing edge-id order (n_crit[0]-1 of
 *        them for a grid, plus the essential class written to *d0_essential).
 *   d2   [cap2] out: D2 pairs in increasing triangle-id order (n_crit[3]).
 *   n_out [2] int64 out: numbers of D0 and D2 pairs (capacity errors as in
 *        dms_critical).
 *   ws   at least dms_diagram_workspace_size(d, n_crit) bytes (it includes
 *        one 32-bit word per tetrahedron id, 24 bytes per vertex).
 * This call synchronises `stream` between pairing rounds (it reads the
 * number of live saddles on the host).
 */
size_t dms_diagram_workspace_size(dms_dims d, const int64_t* n_crit);
int dms_diagram_d0d2(const float* f, const uint32_t* order, const uint8_t* desc,
                     const uint64_t* rec, dms_dims d, const int64_t* crit0,
                     const int64_t* crit1, const int64_t* crit2, const int64_t* crit3,
                     const int64_t* n_crit, dms_pair* d0, int64_t cap0, dms_pair* d2,
                     int64_t cap2, dms_pair* d0_essential, int64_t* n_out, void* ws,
                     size_t ws_bytes, int32_t* dstatus, void* stream);

/* dms_diagram_d0d2_selfcorrecting -- the same D0 / D2 pairs (same arguments,
 * workspace and outputs as dms_diagram_d0d2), paired by the paper's
 * self-correcting pairing (Sec. 4.3, Alg. 4) run as a fixpoint instead of
 * the spanning forest and exact rounds: every round, every saddle of the
 * extremum graph computes the representatives of its two ends by following
 * only links that earlier saddles (in Alg. 1's order) assigned -- each
 * extremum's representative records the saddle that assigned it -- and the
 * younger representative dies at the earliest saddle that claims it
 * (atomicMin); wrong claims from stale links are corrected in later rounds.
 * The rounds stop when no link changes; the result is Alg. 1's.  A chain of
 * components that Alg. 1 merges one by one takes one round per merge; past
 * 65536 rounds the call returns DMS_ERR_TIMEOUT.  Synchronises `stream`
 * once per round (it reads the number of changed links on the host).
 */
int dms_diagram_d0d2_selfcorrecting(const float* f, const uint32_t* order, const uint8_t* desc,
                                    const uint64_t* rec, dms_dims d, const int64_t* crit0,
                                    const int64_t* crit1, const int64_t* crit2,
                                    const int64_t* crit3, const int64_t* n_crit, dms_pair* d0,
                                    int64_t cap0, dms_pair* d2, int64_t cap2,
                                    dms_pair* d0_essential, int64_t* n_out, void* ws,
                                    size_t ws_bytes, int32_t* dstatus, void* stream);

/* ----------------------------------------------------------------- (D1) ---
 * dms_diagram_d1 -- the saddle-saddle pairs D1 of a 3D field (Sec. 2.5 "D1
 * pairing", Alg. 2 and Alg. 3), computed after D0 and D2: the critical
 * triangles that D2 left unpaired are paired with the critical edges that D0
 * left unpaired by homologous propagation.  The boundary of each triangle
 * (a max-heap of edges under the lexicographic key, Z2 by lazy
 * cancellation, kept in a pool of device memory) is expanded at its highest
 * edge through the gradient until that edge is critical; a column whose
 * highest critical edge an earlier triangle settled on adds that triangle's
 * boundary and goes on, the others claim their edge (the earliest triangle
 * wins); all columns work at once, in rounds, until every column is settled
 * on a distinct edge.  The result is the pairing of the sequential Alg. 3.
 *   f, order, rec   as above (desc is not needed).
 *   crit1, crit2    critical edges / triangles from dms_critical (sorted);
 *                   n_crit HOST [4] their counts (n_crit[1], n_crit[2] < 2^32 - 1).
 *   d0, n_d0        the D0 pairs of dms_diagram_d0d2 (n_d0 of them, count on
 *                   the host); d2, n_d2 the D2 pairs.
 *   d1   [cap1] out: D1 pairs (birth = edge, death = triangle) in increasing
 *        triangle-id order (n_crit[2] - n_d2 of them); n_out [1] int64 out
 *        (capacity errors as in dms_critical).
 *   pool_entries  16-byte heap entries of the boundary pool (0: 256 per
 *        critical triangle + 65536; at least 16 per critical triangle).  The
 *        pool is a bump allocator: a heap that grows moves to a new segment
 *        twice its size and its old one is not reused.  A boundary that
 *        outgrows the pool sets (1 << DMS_ERR_CAPACITY) and the call can be
 *        repeated with more (from the start: the rounds before are lost).
 *   ws   at least dms_diagram_d1_workspace_size(d, n_crit, pool_entries).
 * Synchronises `stream` once per round; past 4096 rounds it returns
 * DMS_ERR_TIMEOUT.
 */
size_t dms_diagram_d1_workspace_size(dms_dims d, const int64_t* n_crit, int64_t pool_entries);
int dms_diagram_d1(const float* f, const uint32_t* order, const uint64_t* rec, dms_dims d,
                   const int64_t* crit1, const int64_t* crit2, const int64_t* n_crit,
                   const dms_pair* d0, int64_t n_d0, const dms_pair* d2, int64_t n_d2,
                   dms_pair* d1, int64_t cap1, int64_t* n_out, int64_t pool_entries, void* ws,
                   size_t ws_bytes, int32_t* dstatus, void* stream);

/* ---------------------------------------------------------------- batch ---
 * dms_batch_diagrams -- (i)-(iv) for many fields of uneven dims at once
 * (the batch processing the paper contrasts with its per-dataset runs,
 * Sec. 2.6): one segmented order sort, one persistent gradient kernel whose
 * CTAs take tiles of all fields from a shared queue, one compaction, one set
 * of pairing rounds over the disjoint union of the fields' extremum graphs.
 * Nothing synchronises the host, so the whole call can be captured in a CUDA
 * graph and replayed.
 *   f            concatenated float32 fields (sum of the fields' sizes).
 *   fields_host  [nfields] table (host), fields_dev the same table on the
 *                device (both read during the call).
 *   tile_variant gradient variant, 0..dms_batch_tile_variants()-1: tile shape
 *                variant % 3 (32 x 24, 32 x 16, 32 x 32 anchors per CTA) and
 *                lanes per vertex 1 + variant / 3 (two: the lane pair splits
 *                the rank comparisons, link edges and tet keys of a vertex);
 *                an autotuner picks one; all give the same results.
 *   order, desc, rec  concatenated outputs as in dms_order/dms_gradient, each
 *                field with its own local order and records.
 *   caps         host [4]: capacity, over all fields, of the critical lists
 *                (kept in the workspace); cap_pairs: capacity of d0 and of d2.
 *   d0, d2       pairs with ids and vertex indices LOCAL to their field, in
 *                field order (then saddle-id order); pair_offsets [2][nfields+1]
 *                (device) delimit each field's pairs; d0_essential [nfields].
 *   counts       device [6]: critical simplices per dimension, then the
 *                numbers of D0 and D2 pairs (a count above its capacity sets
 *                (1 << DMS_ERR_CAPACITY); the call can then be repeated with
 *                larger capacities).
 *   ws           at least dms_batch_workspace_size(...) bytes.
 * The spanning forest takes a fixed 40 Boruvka rounds (enough: the active
 * components at least halve per round); the pairing runs
 * dms_batch_max_rounds() exact rounds and finishes the saddles still live
 * in increasing weight (Alg. 1's own order): up to 4096 of them in one CTA,
 * more after a device-wide sort by one thread, which is slow when very many
 * are left (a chain of components that the exact rounds merge one per
 * round) but exact.
 */
int32_t dms_batch_tile_variants(void);
int32_t dms_batch_max_rounds(void);
size_t dms_batch_workspace_size(const dms_field_desc* fields_host, int32_t nfields,
                                const int64_t* caps, int64_t cap_pairs);
int dms_batch_diagrams(const float* f, const dms_field_desc* fields_host,
                       const dms_field_desc* fields_dev, int32_t nfields, int32_t tile_variant,
                       uint32_t* order, uint8_t* desc, uint64_t* rec, const int64_t* caps,
                       int64_t cap_pairs, dms_pair* d0, dms_pair* d2, int64_t* pair_offsets,
                       dms_pair* d0_essential, int64_t* counts, void* ws, size_t ws_bytes,
                       int32_t* dstatus, void* stream);

/* ------------------------------------------------------------------ diff ---
 * dms_backward -- gradient of a loss on diagram values with respect to the
 * field.  A pair sits at (f(birth simplex), f(death simplex)), f(s) being the
 * value of the highest vertex of s (Sec. 2.4); the pairing depends on the
 * order of the values only, so it is locally constant and
 *   dL/df[v] = sum_i g[i][0] [birth_vtx_i == v] + g[i][1] [death_vtx_i == v].
 *   pairs  [n] dms_pair from dms_diagram_d0d2 (D0, D2 or the essential class;
 *          a pair with death_id < 0 contributes its birth term only).
 *   g      [n][2] float32: dL/dbirth, dL/ddeath of each pair.
 *   grad   [N] float32, ACCUMULATED into (zero it first).  Pairs sharing a
 *          carrier vertex are added with float atomics in no fixed order.
 * A carrier outside the grid sets (1 << DMS_ERR_ARG) in *dstatus.
 */
int dms_backward(const dms_pair* pairs, int64_t n, const float* g, dms_dims d, float* grad,
                 int32_t* dstatus, void* stream);

/* -------------------------------------------------------------------- 2D ---
 * The same path on a 2D grid (nx x ny, each >= 2, nx*ny < 2^32 - 1), where
 * the extremum-saddle pairs D0 and D1 are the whole persistence diagram.
 * Conventions as above, one dimension down: vertex v = x + nx*y; the
 * Freudenthal split of every square along its (1,1) diagonal; ids (int64)
 *   vertex v;  edge 3a + k, corner {+x, +y, +x+y}[k];
 *   triangle 2a + k = {a, a+p, a+(1,1)}, p = {+x, +y}[k].
 * Neighbour slots of a vertex: s < 3 -> +corner, s >= 3 -> -corner of edge
 * type s % 3.
 *
 * dms2_order -- as dms_order (Sec. 2.1), on nx*ny vertices.
 * dms2_gradient -- ProcessLowerStars on every vertex (Sec. 2.3); y is tiled
 *   by 16 rows in the launch's second dimension, so ny is at most
 *   16 * 65535 = 1,048,560 (a taller grid returns DMS_ERR_CUDA):
 *   desc  [n] uint8 out: 0..5 the slot of the edge v is paired with, 15 a minimum.
 *   rec   [n] uint16 out, per anchor a: bits 3k..3k+2 edge k (0 = absent or
 *         paired with its top vertex, 1..2 = paired with the (code-1)-th
 *         triangle holding it by increasing id on the unbounded lattice,
 *         7 = critical); bits 9+3k..11+3k triangle k (0 = absent, 1..3 =
 *         paired with the facet that omits vertex (code-1) of its chain
 *         a < a+p < a+(1,1), 7 = critical); other bits 0.
 * dms2_critical -- the critical vertices, edges and triangles in increasing
 *   id order (caps, counts and errors as dms_critical, three lists).
 * dms2_diagram_d0d1 -- D0 as in 3D (Alg. 1, minima against edges); D1 by
 *   the dual walks from the two triangles of every critical edge to a
 *   critical triangle or OUTSIDE (off the grid), edges taken in decreasing
 *   order, the lower maximum dying (Alg. 1 on the dual graph).  D0 pairs in
 *   increasing edge-id order (n_crit[0]-1 of them, plus the essential class),
 *   D1 pairs (birth = edge, death = triangle) in increasing edge-id order
 *   (n_crit[2] of them).  n_crit is a HOST array of 3 (n_crit[1] < 2^30).
 *   Synchronises the stream between pairing rounds, as dms_diagram_d0d2.
 */
size_t dms2_order_workspace_size(int32_t nx, int32_t ny);
int dms2_order(const float* f, int32_t nx, int32_t ny, uint32_t* order, void* ws, size_t ws_bytes,
               int32_t* dstatus, void* stream);
int dms2_gradient(const uint32_t* order, int32_t nx, int32_t ny, uint8_t* desc, uint16_t* rec,
                  void* stream);
size_t dms2_critical_workspace_size(int32_t nx, int32_t ny);
int dms2_critical(const uint8_t* desc, const uint16_t* rec, int32_t nx, int32_t ny, int64_t* crit0,
                  int64_t* crit1, int64_t* crit2, const int64_t* cap, int64_t* counts, void* ws,
                  size_t ws_bytes, int32_t* dstatus, void* stream);
size_t dms2_diagram_workspace_size(int32_t nx, int32_t ny, const int64_t* n_crit);
int dms2_diagram_d0d1(const float* f, const uint32_t* order, const uint8_t* desc,
                      const uint16_t* rec, int32_t nx, int32_t ny, const int64_t* crit0,
                      const int64_t* crit1, const int64_t* crit2, const int64_t* n_crit,
                      dms_pair* d0, int64_t cap0, dms_pair* d1, int64_t cap1,
                      dms_pair* d0_essential, int64_t* n_out, void* ws, size_t ws_bytes,
                      int32_t* dstatus, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DMS_H_ */
