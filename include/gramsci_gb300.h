/*
 * gramsci_gb300.h - C ABI of the GB300 (sm_103a) query engine for binned
 * 3-point and 4-point correlation tuple counts over a fixed-radius graph,
 * after GRAMSCI v2 (Sabiu, "Fast Graph-based Higher-Order Clustering
 * Statistics on the GPU").
 *
 * Conventions shared by every call
 * --------------------------------
 * Coordinates are int32 lattice coordinates in units of 1/1024 h^-1 Mpc
 * (gs_quantize makes them from float positions). A periodic box has side
 * box_u > 0 lattice units and displacements use the minimum image
 * (2d >= box_u: d -= box_u; 2d < -box_u: d += box_u); box_u == 0 selects an
 * open box. Radial bins are given by nb+1 strictly increasing integer edges
 * E_0 < ... < E_nb (lattice units); a pair with squared distance D2 is an
 * edge iff E_0^2 <= D2 < E_nb^2 and its bin is the largest b with
 * E_b^2 <= D2 (Sec. 2.1).
 *
 * Pointers: every array argument may be host or device memory (the library
 * asks the CUDA runtime which). Inputs are owned by the caller and never
 * retained after the call returns. Outputs are allocated by the caller,
 * overwritten (not accumulated) and complete when the call returns: every
 * call synchronises options->stream before returning.
 *
 * Streams: all device work of a call is queued on options->stream (a
 * cudaStream_t; NULL = the legacy default stream). options may be NULL,
 * which means all fields zero.
 *
 * Output order: configuration index = rank of the configuration's canonical
 * representative in lexicographic order. 3-point: sorted bin triples
 * (r1 <= r2 <= r3), C(nb+2, 3) of them (Sec. 5.1). 4-point: S4 orbits of the
 * edge-bin tuple (b01, b02, b03, b12, b13, b23) represented by their
 * lexicographically smallest member (Sec. 5.2); gs_config_bins lists them.
 *
 * Status: 0 on success, else one of the negative GS_E* codes below; on
 * error the outputs are unspecified, nothing stays allocated and the
 * library remains usable. gs_strerror gives a message.
 */
#ifndef GRAMSCI_GB300_H
#define GRAMSCI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GS_OK = 0,
  GS_EINVAL = -1,       /* NULL where an array is required, nb < 1, bad flag */
  GS_ERANGE = -2,       /* value outside the supported range (see each call) */
  GS_ENOMEM = -3,       /* allocation failed, or the device budget is too small */
  GS_ECUDA = -4,        /* a CUDA runtime call or kernel launch failed */
  GS_ETIMEOUT = -5,     /* a bounded device-side wait expired */
  GS_EUNSUPPORTED = -6  /* weights whose exact weighted sums would not fit */
};

/* Opaque device-resident neighbour graph, owned by the library. */
typedef struct gs_graph gs_graph;

typedef struct {
  /* Device-memory cap for the graph's edge storage in bytes; 0 = no cap.
   * A graph above the cap keeps its edges in pinned host memory and every
   * query streams row windows through device buffers (out-of-core mode). */
  uint64_t device_budget_bytes;
  /* > 0 forces that many row windows (out-of-core mode even when the
   * graph fits); 0 = automatic. */
  int32_t force_windows;
  /* Kernel variant bits: 0 = automatic (gs_count_3pcf tests every pair of
   * a hub's neighbours geometrically; see gs_count_3pcf). 512 = gs_count_3pcf
   * uses the merge-walk kernel of Sec. 3.1 instead, as does any of the bits
   * 1, 2, 8, 16, 32 and 64, which select its paths. 1 = exercise the
   * long-row code paths on any input (the walk probes a hash of the hub row
   * staged in 64-word segments; gs_count_4pcf* keeps every hub's workspace in
   * global memory; gs_build_graph tests candidate pairs in 64-bit arithmetic
   * even where 32 bits suffice). 2 = the walk reads hub rows from global memory
   * instead of staging them. 4 = gs_count_3pcf computes configuration
   * indices instead of looking them up in a shared table, and
   * gs_count_4pcf* bins the non-hub edges by binary search over the bin
   * edges instead of squared-distance buckets. 8 = gs_count_3pcf
   * limits its direct-address table to 2 KB (rows split at their largest id
   * gap, or hashed), and gs_count_4pcf* keeps only 64 orbits' counters
   * in shared memory (the others go straight to the global counts and
   * sums). 16 = gs_count_3pcf gives each block's first staging
   * wait no polls, so the call fails with GS_ETIMEOUT after the blocks have
   * let their copies land (tests of the failure path). 32 = weighted
   * gs_count_3pcf compacts each warp's hits before recording them. 64 =
   * gs_count_3pcf streams spoke rows through a per-warp ring of
   * asynchronous copies (deeper prefetch). Other results are identical;
   * the bits exist for testing and tuning. */
  int32_t variant;
  /* cudaStream_t for all device work; NULL = legacy default stream. */
  void* stream;
  /* Reserved, must be 0. */
  uint32_t flags;
  /* Hub sharding for multi-GPU splits of one catalogue: with shards > 1 a
   * query counts only the tuples whose smallest internal label lies in the
   * shard-th of `shards` contiguous hub ranges of about equal edge count;
   * the sum over shard = 0 .. shards-1 is the full result (integer counts
   * and exact weighted sums add exactly). shards <= 1 counts everything. */
  int32_t shard;
  int32_t shards;
  /* NULL, or receives the device time in milliseconds of the call's main
   * kernel launches (the counting kernels of gs_count_*, the two row passes
   * of gs_build_graph, the pair sweep of gs_disconnected_4pcf), measured
   * with CUDA events on options->stream. */
  double* kernel_ms;
} gs_options;

/* Graph statistics (host struct filled by gs_graph_info). */
typedef struct {
  int64_t n;               /* points */
  int32_t nb;              /* radial bins */
  int32_t max_degree;      /* largest |N+(i)| */
  int64_t edges;           /* unordered edges = sum_i |N+(i)| */
  int64_t edge_slots;      /* stored edge words including row padding */
  int64_t probe_words;     /* sum over edges (i,j), i<j, of |N+(j)| */
  int64_t bytes_per_edge;  /* bytes of one stored edge word (4 or 8) */
  int64_t device_bytes;    /* device bytes held by the graph */
  int32_t windows;         /* row windows (1 = fully resident) */
  int32_t cells;           /* cells per axis of the build grid (x) */
  int64_t walk_words;      /* sum over edges (i,j), i<j, of the words of N+(j)
                              up to the largest id of N+(i): what a merge-walk
                              of the spoke row reads before the hub row is
                              exhausted (Sec. 3.1) */
} gs_graph_stats;

/*
 * gs_quantize - positions in h^-1 Mpc to lattice coordinates (the input
 * step of Sec. 2.1). X = floor(1024 x) per axis; periodic (periodic != 0)
 * wraps X modulo box_u, otherwise X must lie in [0, box_u).
 *   pos  float64 [n][3] (row-major), xyz int32 [n][3] out.
 * Errors: GS_EINVAL (NULL, n < 0, box_u <= 0), GS_ERANGE (an open-box
 * coordinate outside [0, box_u), or box_u >= 2^31).
 */
int gs_quantize(const double* pos, int64_t n, int64_t box_u, int periodic, int32_t* xyz,
                const gs_options* options);

/*
 * gs_build_graph - radius-search graph of Sec. 2.1 (Eq. adjacency) built on
 * the device with a cell list. The library relabels points in cell order;
 * outputs of every query are invariant under relabelling.
 *   xyz      int32 [n][3] lattice coordinates (periodic: in [0, box_u);
 *            open: in [0, 2^30)).
 *   box_u    periodic box side in lattice units, 0 = open box.
 *   edges_u  int64 [nb+1] strictly increasing bin edges, E_0 >= 0.
 *   out      receives the new graph; release it with gs_free_graph.
 * Errors: GS_EINVAL (NULL, n < 0, nb < 1), GS_ERANGE (nb > 254, edges not
 * strictly increasing, E_nb >= 2^19, 4 E_nb >= box_u for a periodic box,
 * n >= 2^31, a coordinate out of range), GS_ENOMEM.
 */
int gs_build_graph(const int32_t* xyz, int64_t n, int64_t box_u, const int64_t* edges_u, int nb,
                   const gs_options* options, gs_graph** out);

/* gs_graph_info - fill *stats (host pointer). */
int gs_graph_info(const gs_graph* g, gs_graph_stats* stats);

/*
 * gs_graph_tri_words - statistics of the triangle walk that bound the
 * 4-point query's memory traffic (the three-way merge of Eq. threeway reads,
 * for every triangle i < j < k, the row N+(k) of its largest vertex):
 *   *triangles   number of triangles (every configuration together);
 *   *tail_words  sum over those triangles of |N+(k)|.
 * Host pointers. Runs a plain binary-search walk over the graph (seconds
 * for graphs of about 1e8 edges). Errors: GS_EINVAL, GS_ENOMEM, GS_ECUDA.
 */
int gs_graph_tri_words(const gs_graph* g, int64_t* triangles, int64_t* tail_words);

/*
 * gs_graph_export - copy the oriented CSR out, in the graph's own labels.
 *   ptr  int64 [n+1]: row i holds N+(i) = {j > i adjacent to i} in
 *        nbr[ptr[i] .. ptr[i]+deg(i)) in ascending order (rows are padded,
 *        so ptr[i+1]-ptr[i] may exceed deg(i)).
 *   deg  int32 [n], nbr int32 [edge_slots], bin uint8 [edge_slots],
 *   perm int32 [n]: perm[k] = caller index of internal label k.
 * Any output may be NULL. Host or device pointers.
 */
int gs_graph_export(const gs_graph* g, int64_t* ptr, int32_t* deg, int32_t* nbr, uint8_t* bin,
                    int32_t* perm);

/*
 * gs_count_3pcf - binned triangle counts (Sec. 2.2). Every triangle i<j<k
 * is found at its smallest vertex i from the pair (j, k) of N+(i); the
 * default kernel decides whether (j, k) is an edge from the exact lattice
 * distance of the pair, the merge-walk kernel (variant bit 512) by the
 * hub-and-spoke intersection of sorted rows of Sec. 3.1. Both give the
 * same counts and sums.
 *   w       NULL (unweighted) or float32 [n] weights in caller order.
 *   counts  uint64 [C(nb+2,3)] triangle counts per configuration.
 *   wsum    NULL or float64 [C(nb+2,3)]: sum of w_i w_j w_k per
 *           configuration, accumulated exactly and rounded once to the
 *           nearest double (ties to even). Weights whose magnitudes span
 *           more than about 2^5 are split exactly (W = A + 2^27 B) and the
 *           sums of four exact evaluations interpolated: four launches.
 * Errors: GS_EINVAL, GS_EUNSUPPORTED (weights not finite, or magnitudes
 * spanning more than about 2^28), GS_ETIMEOUT, GS_ECUDA.
 */
int gs_count_3pcf(const gs_graph* g, const float* w, uint64_t* counts, double* wsum,
                  const gs_options* options);

/*
 * gs_tune_3pcf - autotuner for gs_count_3pcf. Times the launch variants
 * (hub rows staged in shared memory or read from global memory;
 * configuration indices computed or looked up) on one hub shard of g
 * (about 1/16 of its edges, weighted like w) and remembers the fastest for
 * graphs with the same nb, weight mode and degree class; calls with
 * options->variant = -1 then use it (0 when nothing was tuned).
 * *best_variant receives the choice. Errors: as gs_count_3pcf.
 */
int gs_tune_3pcf(const gs_graph* g, const float* w, const gs_options* options,
                 int32_t* best_variant);

/*
 * gs_count_3pcf_noalloc - unweighted gs_count_3pcf that allocates nothing.
 * The paper has no counterpart: this entry point is for callers that may
 * not let a library allocate memory during a call (a process that gave all
 * device memory to its own pool, so that any further allocation fails; a
 * real-time loop that must avoid the allocator's locks and the device
 * synchronisation that cudaFree implies). Instead of allocating, it
 * uses one fixed 64 KB scratch array compiled into the library, which every
 * GPU that loads the library holds until the process exits.
 *   g       a resident graph (not out-of-core), nb <= 35.
 *   counts  uint64 [C(nb+2,3)], host or device; identical to gs_count_3pcf
 *           for every options->variant (-1 = the tuned variant).
 * The first call on each device looks up the scratch array's device address
 * (with that device current); make that first call before any stream
 * capture. All calls share the array and it keeps the last call's contents:
 * each call clears what must start at zero, but calls whose device work
 * overlaps (different streams or host threads) race and give wrong results.
 * options->kernel_ms, shard and shards are ignored.
 * Errors: GS_EINVAL (NULL, out-of-core graph), GS_ERANGE (nb > 35, or more
 * than 64 devices), GS_ETIMEOUT, GS_ECUDA.
 */
int gs_count_3pcf_noalloc(const gs_graph* g, uint64_t* counts, const gs_options* options);

/*
 * gs_count_3pcf_batch - gs_count_3pcf for many catalogues in one
 * persistent launch: the hubs of all graphs form one work queue, so small
 * catalogues share the GPU instead of each paying a launch and a tail.
 * Results are identical to one gs_count_3pcf call per graph.
 *   graphs   n_graphs resident graphs (not out-of-core) with equal nb.
 *   w        NULL (all unweighted) or n_graphs weight arrays (none NULL).
 *   counts   n_graphs output arrays of C(nb+2,3) uint64.
 *   wsum     NULL or n_graphs arrays (an entry may be NULL) of float64.
 * Errors: GS_EINVAL (NULL entries, unequal nb, out-of-core graph), and as
 * gs_count_3pcf.
 */
int gs_count_3pcf_batch(const gs_graph* const* graphs, int32_t n_graphs, const float* const* w,
                        uint64_t* const* counts, double* const* wsum, const gs_options* options);

/*
 * Recorded batched launches. gs_plan_3pcf_batch records one unweighted
 * batched 3pCF count of fixed resident graphs (clearing the outputs and the
 * persistent kernel) into a CUDA graph; gs_plan_launch replays it on a
 * stream, asynchronously, with no allocation and no host synchronisation;
 * gs_plan_wait synchronises the stream and returns GS_ETIMEOUT if the last
 * replay's kernel reported an expired wait. The graphs must outlive the
 * plan; counts are n_graphs DEVICE arrays of C(nb+2,3) uint64 rewritten by
 * every replay. Replays of one plan must not overlap each other on the GPU.
 * Errors: GS_EINVAL (NULL, unequal nb, out-of-core graph, host outputs),
 * GS_ENOMEM, GS_ECUDA.
 */
typedef struct gs_plan gs_plan;
int gs_plan_3pcf_batch(const gs_graph* const* graphs, int32_t n_graphs, uint64_t* const* counts,
                       const gs_options* options, gs_plan** out);
int gs_plan_launch(gs_plan* plan, void* stream);
int gs_plan_wait(gs_plan* plan, void* stream);
void gs_plan_destroy(gs_plan* plan);

/*
 * gs_count_3pcf_equilateral - equilateral 3pCF (named among the GPU query
 * kernels in Sec. 3.5 and Sec. 4.8; the paper gives no definition). Here it
 * is the nb configurations whose three sides share one bin: counts[b] is the
 * number of triangles with all three pair separations in bin b, equal to the
 * full 3pCF's entry at configuration (b, b, b). The default kernel groups
 * each hub's neighbours by hub-edge bin and tests only the pairs within a
 * group; options->variant bit 512 selects the merge-walk's instantiation,
 * which follows same-bin edges only.
 *   w       NULL or float32 [n] weights (caller's order).
 *   counts  uint64 [nb]; wsum NULL or float64 [nb] (exact sums of
 *           w_i w_j w_k rounded once; needs w).
 * Host or device pointers; options->shard/shards split the hubs as for
 * gs_count_3pcf. Errors: as gs_count_3pcf.
 */
int gs_count_3pcf_equilateral(const gs_graph* g, const float* w, uint64_t* counts, double* wsum,
                              const gs_options* options);

/*
 * gs_count_3pcf_mu - anisotropic 3pCF. The paper's conclusions name mu
 * binning for redshift-space distortions without defining it; the reading
 * here: the line of sight is the z axis (distant observer), a triangle's
 * mu is |n_z| / |n| for the normal n of its plane (the same from every
 * vertex), its bin m the largest in [0, nmu) with m / nmu <= mu (decided in
 * exact integer arithmetic; mu = 1 falls in bin nmu - 1), and collinear
 * triangles (n = 0) go to bin nmu. Summing over the nmu + 1 bins gives
 * gs_count_3pcf.
 *   w       NULL or float32 [n] weights (caller's order); magnitudes must
 *           span at most about 2^5 (GS_EUNSUPPORTED otherwise).
 *   nmu     1..64 mu bins.
 *   counts  uint64 [C(nb+2,3)][nmu + 1], configuration-major as in
 *           gs_count_3pcf; wsum NULL or float64 of the same shape (exact
 *           sums of w_i w_j w_k rounded once; needs w).
 * Host or device pointers; options->shard/shards split the hubs as for
 * gs_count_3pcf. Errors: GS_EINVAL (NULL graph or counts, wsum without w,
 * nmu outside 1..64), and as gs_count_3pcf.
 */
int gs_count_3pcf_mu(const gs_graph* g, const float* w, int32_t nmu, uint64_t* counts,
                     double* wsum, const gs_options* options);

/*
 * gs_count_4pcf - binned tetrahedron counts (Sec. 2.2, Sec. 3.1.1):
 * tetrahedra whose six pairs are all edges, one count per S4 orbit.
 *   counts uint64 [n_orbits], wsum NULL or float64 [n_orbits] (exact;
 *   weights spanning more than about 2^5: five launches, as for the 3pCF).
 * Errors: as gs_count_3pcf (the weight span limit is about 2^26); GS_ERANGE
 * when nb > 16.
 */
int gs_count_4pcf(const gs_graph* g, const float* w, uint64_t* counts, double* wsum,
                  const gs_options* options);

/*
 * gs_count_4pcf_parity - parity-decomposed 4pCF (Sec. 3.2, Eq. volume).
 * For each tetrahedron V = (r_01 x r_02) . r_03 is evaluated exactly in
 * integers in the vertex order that maps it onto its orbit representative.
 *   even  uint64 [n_orbits]: every tetrahedron (equals gs_count_4pcf).
 *   odd   int64 [n_orbits]: sum of sign(V) over tetrahedra with V != 0 in
 *         chiral orbits (orbits whose representative no odd permutation
 *         fixes); zero for achiral orbits. Degenerate tetrahedra (V == 0)
 *         add nothing to odd.
 *   weven, wodd: NULL or float64 [n_orbits], the same with weights.
 * Errors: as gs_count_4pcf.
 */
int gs_count_4pcf_parity(const gs_graph* g, const float* w, uint64_t* even, int64_t* odd,
                         double* weven, double* wodd, const gs_options* options);

/*
 * gs_count_4pcf_parity_pix - parity 4pCF with pixelised spoke directions
 * (Sec. 3.2: the direction of each spoke is quantised to a pixel on the
 * unit sphere, one byte per edge, and tetrahedra whose pixel volume is below
 * 1e-9 in magnitude are degenerate and left out of the odd channel). The
 * pixel scheme, which the paper leaves open, is fixed here as 256 equal-area
 * pixels (see gs_direction_pixels). For each tetrahedron the three spokes
 * run from its vertex with the smallest caller index to the other three in
 * ascending caller index; V is (u1 x u2) . u3 of their pixel centres in
 * FP64; odd gets sign(V) times the parity of the relabelling onto the orbit
 * representative when the orbit is chiral and |V| >= 1e-9; a spoke of zero
 * length (coincident points) makes the tetrahedron degenerate.
 *   even, weven: as gs_count_4pcf_parity (identical values).
 *   odd, wodd:   the pixelised odd channel.
 * Errors: as gs_count_4pcf_parity.
 */
int gs_count_4pcf_parity_pix(const gs_graph* g, const float* w, uint64_t* even, int64_t* odd,
                             double* weven, double* wodd, const gs_options* options);

/*
 * gs_direction_pixels - the direction pixel of gs_count_4pcf_parity_pix for
 * integer vectors (Sec. 3.2's pixel byte): 16 bands of width 1/8 in
 * cos(theta) = z / |d| on [-1, 1] times 16 sectors of pi/8 in
 * phi = atan2(y, x) in [0, 2 pi); a direction on a band or sector edge
 * belongs to the band or sector above it; sector 0 on the z axis; pixel =
 * 16 band + sector. Decided exactly on the device: single-precision
 * estimates with error bounds, confirmed by integer comparisons near an edge.
 *   dirs    int32 [n][3] nonzero vectors (host or device), |components| < 2^20.
 *   pixels  uint8 [n] out (host or device).
 * Errors: GS_EINVAL, GS_ENOMEM, GS_ECUDA.
 */
int gs_direction_pixels(const int32_t* dirs, int64_t n, uint8_t* pixels, const gs_options* options);

/*
 * gs_disconnected_4pcf - internal 2pCF and disconnected 4pCF on the same
 * graph (Sec. 3.3, Eq. disc), one sweep over the edges.
 *   w          NULL or float32 [n] weights (pair sums use w_i w_j, exact).
 *   rr         NULL: analytic random pairs of a periodic box,
 *              RR[b] = P (4 pi / 3)(E_{b+1}^3 - E_b^3) / box_u^3 with
 *              P = n(n-1)/2, or ((sum w)^2 - sum w^2)/2 with weights;
 *              else float64 [nb] random pair counts supplied by the caller.
 *   pairs      NULL or uint64 [nb] unordered edge counts per bin.
 *   xi         NULL or float64 [nb]: pair sum / RR - 1.
 *   zeta_disc  NULL or float64 [n_orbits]: xi(r01) xi(r23) + xi(r02) xi(r13)
 *              + xi(r03) xi(r12) on each orbit representative, FP64, left to
 *              right, no fused multiply-add.
 * Errors: GS_EINVAL (rr NULL for an open box), GS_ERANGE (zeta_disc with
 * nb > 16), GS_EUNSUPPORTED, GS_ECUDA.
 */
int gs_disconnected_4pcf(const gs_graph* g, const float* w, const double* rr, uint64_t* pairs,
                         double* xi, double* zeta_disc, const gs_options* options);

/*
 * gs_connected_4pcf - connected 4pCF with the signed-weight estimator
 * (Sec. 2.1 weights, Sec. 3.3, Eq. disc, Eq. conn). One weighted pair
 * sweep and one weighted parity 4pCF pass over each of two graphs built on
 * the same bin edges:
 *   g_dr      graph of the union of data and randoms.
 *   w_signed  float32 [n of g_dr], in g_dr's input order: data weights
 *             (normalised by the caller to sum +1) and random weights
 *             (normalised to sum -1). The signed pair sum of a bin is then
 *             the Landy-Szalay numerator DD - 2DR + RR.
 *   g_r       graph of the randoms alone.
 *   w_r       float32 [n of g_r]: the random weights with the sign of a
 *             data weight (normalised to sum +1); they give RR and RRRR.
 * Outputs (each NULL or float64, host or device memory):
 *   xi         [nb]       signed pair sum / RR (no constant subtracted).
 *   zeta_even  [n_orbits] signed quadruplet sum / RRRR, even channel.
 *   zeta_odd   [n_orbits] signed parity-odd quadruplet sum / RRRR.
 *   zeta_disc  [n_orbits] xi(r01) xi(r23) + xi(r02) xi(r13) + xi(r03) xi(r12)
 *              on each orbit representative.
 *   zeta_conn  [n_orbits] zeta_even - zeta_disc; the odd channel is
 *              connected as it stands and is not corrected.
 * All sums are exact fixed-point sums rounded once to FP64; every ratio,
 * product and sum above is one IEEE-rounded FP64 operation, left to right,
 * without fused multiply-add. A bin or orbit with RR or RRRR zero yields
 * the IEEE quotient (inf or NaN).
 * Errors: GS_EINVAL (a NULL graph or weight array, different bin edges,
 * options->shards > 1: ratios do not add over hub shards), GS_ERANGE
 * (nb > 16), GS_EUNSUPPORTED (non-finite weights, or weights of one graph
 * whose nonzero magnitudes span more than the exact fixed-point range,
 * about a factor 2^5), GS_ENOMEM, GS_ETIMEOUT, GS_ECUDA.
 */
int gs_connected_4pcf(const gs_graph* g_dr, const float* w_signed, const gs_graph* g_r,
                      const float* w_r, double* xi, double* zeta_even, double* zeta_odd,
                      double* zeta_disc, double* zeta_conn, const gs_options* options);

/*
 * gs_config_mask_cm - Cayley-Menger realisability of the 4pCF orbits
 * (Sec. 5.2): an orbit is kept when the six bin centres of its
 * representative, taken as edge lengths, give a positive Cayley-Menger
 * determinant (288 V^2 > 0), i.e. form a non-degenerate tetrahedron.
 *   nb         1..16 bins; edges_u int64 [nb+1] host, strictly increasing,
 *              edges_u[0] >= 0, edges_u[nb] <= 2^19 (512 h^-1Mpc).
 *   mask       uint8 [n_orbits] (host or device): 1 kept, 0 excluded.
 *   n_realisable  NULL or receives the number kept.
 * The bin centre is the midpoint (E_b + E_{b+1}) / 2; the determinant's sign
 * is evaluated exactly (128-bit integers on doubled centres).
 * Errors: GS_EINVAL, GS_ERANGE, GS_ENOMEM, GS_ECUDA.
 */
int gs_config_mask_cm(int nb, const int64_t* edges_u, uint8_t* mask, int64_t* n_realisable,
                      const gs_options* options);

/*
 * gs_rebin_3pcf - exact fine-to-coarse rebinning of 3pCF results (Sec. 5.1
 * rebins the native fine-bin measurement onto coarser bins).
 *   bin_map    int32 [nb_fine] (host or device): the coarse bin holding each
 *              fine bin, or -1 to drop every configuration using that fine
 *              bin. Coarse bins that unite consecutive fine bins give exactly
 *              the counts a direct count on the coarse edges gives.
 *   counts     NULL or uint64 [C(nb_fine+2,3)] -> coarse_counts uint64
 *              [C(nb_coarse+2,3)] (both NULL or both set).
 *   wsum       NULL or float64 fine -> coarse_wsum float64 coarse.
 * Each coarse configuration sums its fine configurations in ascending fine
 * index (integers exactly, FP64 with one rounding per addition), so results
 * repeat bit for bit. Inputs and outputs may be host or device memory.
 * Errors: GS_EINVAL (NULL map, unpaired arrays, a map value outside
 * [-1, nb_coarse)), GS_ERANGE (nb > 254), GS_ENOMEM, GS_ECUDA.
 */
int gs_rebin_3pcf(int nb_fine, int nb_coarse, const int32_t* bin_map, const uint64_t* counts,
                  const double* wsum, uint64_t* coarse_counts, double* coarse_wsum,
                  const gs_options* options);

/*
 * gs_rebin_4pcf - exact fine-to-coarse rebinning of parity 4pCF results.
 * A fine orbit's representative goes through bin_map in its own vertex
 * labelling and lands in the coarse orbit holding that labelled tuple. Its
 * odd count changes sign when the relabelling onto the coarse representative
 * is an odd permutation (the sign of V follows the vertex order, Sec. 3.2),
 * and is dropped when the coarse orbit is not chiral.
 *   even/c_even uint64, odd/c_odd int64, weven/c_weven and wodd/c_wodd
 *   float64, fine [n_orbits(nb_fine)] -> coarse [n_orbits(nb_coarse)];
 *   each pair both NULL or both set. Summation order as gs_rebin_3pcf.
 * Errors: as gs_rebin_3pcf; GS_ERANGE when a bin count exceeds 16.
 */
int gs_rebin_4pcf(int nb_fine, int nb_coarse, const int32_t* bin_map, const uint64_t* even,
                  const int64_t* odd, const double* weven, const double* wodd, uint64_t* c_even,
                  int64_t* c_odd, double* c_weven, double* c_wodd, const gs_options* options);

/* gs_num_configs - number of configurations: npoint 3 -> C(nb+2,3);
 * npoint 4 -> (nb^6 + 9 nb^4 + 14 nb^2) / 24 (Sec. 5.1, Sec. 5.2).
 * Errors: GS_EINVAL (npoint not 3 or 4, nb < 1), GS_ERANGE (npoint 4 with
 * nb > 16, npoint 3 with nb > 254). */
int gs_num_configs(int npoint, int nb, int64_t* n);

/* gs_config_bins - canonical representative of configuration idx: 3 bins
 * (npoint 3) or 6 bins in slot order (01,02,03,12,13,23) (npoint 4);
 * *chiral (may be NULL) is 1 for chiral 4-point orbits, else 0. Host
 * pointers. Errors: as gs_num_configs, GS_ERANGE for idx out of range. */
int gs_config_bins(int npoint, int nb, int64_t idx, uint8_t* bins, int* chiral);

/* ------------------------------------------------------------------------
 * Request loop (continuous batching of catalogue queries).
 *
 * A server owns two host threads and two CUDA streams on the device that
 * was current at gs_server_create. Requests are admitted in arrival order
 * while the graphs held on the device fit in device_budget_bytes (a request
 * that alone exceeds it runs when nothing else is held); graph builds of
 * admitted requests overlap the counting of earlier ones; ready 3pCF
 * requests with equal nb and weighting are counted together in one batched
 * persistent launch (as gs_count_3pcf_batch); 4pCF requests run the parity
 * kernel one by one. Results are identical to single calls.
 */
typedef struct gs_server gs_server;

typedef struct {
  uint64_t device_budget_bytes; /* graph memory admitted at once; 0 = 80% of free */
  int32_t max_batch;            /* catalogues per batched launch; 0 = 64 */
  int32_t reserved;             /* must be 0 */
} gs_server_config;

typedef struct {
  const int32_t* xyz;     /* [n][3] lattice coordinates (host), copied at submit */
  int64_t n;
  int64_t box_u;          /* periodic side, 0 = open box */
  const int64_t* edges_u; /* [nb+1], copied at submit */
  int32_t nb;
  int32_t npoint;         /* 3: gs_count_3pcf; 4: gs_count_4pcf_parity */
  const float* w;         /* NULL or [n] weights (host), copied at submit */
  /* Outputs: caller-owned HOST arrays that must stay valid until
   * gs_server_wait returns for this ticket. */
  uint64_t* counts;       /* 3pCF counts, or 4pCF even channel */
  int64_t* odd;           /* 4pCF odd channel (required for npoint 4) */
  double* wsum;           /* NULL, or weighted sums (3pCF) / weighted even (4pCF) */
} gs_request;

typedef struct {
  int32_t status;   /* the request's GS_* status */
  double t_submit;  /* seconds since gs_server_create */
  double t_start;   /* admitted (graph build begins) */
  double t_done;    /* results written */
} gs_ticket_info;

int gs_server_create(const gs_server_config* cfg, gs_server** out);
/* Queue a request; *ticket identifies it. Errors: GS_EINVAL. */
int gs_server_submit(gs_server* s, const gs_request* req, int64_t* ticket);
/* Block until the ticket completes (timeout_s < 0: no limit); returns its
 * status, or GS_ETIMEOUT if the wait timed out (the ticket stays valid). */
int gs_server_wait(gs_server* s, int64_t ticket, double timeout_s, gs_ticket_info* info);
/* Finish every queued request, stop the threads, release the server. */
int gs_server_destroy(gs_server* s);

/* gs_kernel_launches - number of CUDA kernels this library has launched in
 * this process (all devices, all threads). */
uint64_t gs_kernel_launches(void);

/* gs_free_graph - release a graph (NULL is ignored). */
void gs_free_graph(gs_graph* g);

/* gs_strerror - static message for a status code. */
const char* gs_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* GRAMSCI_GB300_H */
