/*
 * ffc_gb300.h -- C ABI of the GB300 (sm_103a) tensor-representation library.
 *
 * The library evaluates element tensors of bilinear (and linear) variational forms
 * on affine simplices by the tensor representation A^K_i = A0_{i alpha} G_K^alpha
 * (Kirby & Logg, "A Compiler for Variational Forms", Section 3.2, eq.
 * (tensorproduct)) and adds them into a global CSR matrix (or, for a linear form,
 * a global vector) through the local-to-global dof map (Section 2.2, Algorithm 2).
 *
 * Conventions shared by every entry point
 *  - Return value: FFC_OK (0) or a negative ffc_status. Argument checks happen
 *    before any launch; a call that returns an error launched nothing.
 *  - Pointers marked "device" are caller-owned CUDA device memory on the current
 *    device, contiguous, row-major, 16-byte aligned. Pointers marked "host" are
 *    caller-owned host memory. The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is asynchronous on that stream.
 *  - Local dof order on a simplex with vertices 0..d: for m = 0..d, for each
 *    vertex subset S of size m+1 in lexicographic order, the lattice points with
 *    support exactly S in descending lexicographic order of their barycentric
 *    multi-index (vertices, then edges 01,02,03,12,13,23, faces, interior).
 *    Vector spaces are component blocked: i = c*n_scalar + s.
 *  - Element tensor layout: A_K[e][i1][i2], i1 = test (row), i2 = trial (column),
 *    the dense row-major block of Section 5.5 ("block[]"). A linear form (rank 1)
 *    has A_K[e][i], i = test index: every "n*n" below reads "n" for it.
 *  - Geometry: J = [x_1 - x_0, ..., x_d - x_0] from the cell's vertices in the
 *    given order; G_K uses |det J| (negatively oriented cells are allowed).
 *  - Device-side problems (a degenerate cell, a CSR slot out of range) do not
 *    stop a launch: they set bits in a library-owned device status word that
 *    ffc_status_poll() returns and clears.
 */
#ifndef FFC_GB300_H
#define FFC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffc_form ffc_form;   /* opaque; owns the reference tensor (host and device copies) */
typedef struct ffc_batch ffc_batch; /* opaque; a heterogeneous work list for one persistent launch */
typedef struct ffc_row_plan ffc_row_plan; /* opaque; row-owner view of a dof map (ffc_assemble_rows) */
typedef struct ffc_qform ffc_qform;       /* opaque; a form in the quadrature representation (Section 3.4) */

typedef enum {
  FFC_OK = 0,
  FFC_EINVAL = -1,        /* null pointer, bad size, bad enum value */
  FFC_ENOMEM = -2,        /* host or device allocation failed */
  FFC_ECUDA = -3,         /* a CUDA runtime call failed (message via ffc_last_error) */
  FFC_EDEGENERATE = -4,   /* status word: at least one cell had |det J| <= 1e-14 h_max^d */
  FFC_EUNSUPPORTED = -5,  /* (form, cell, degree, precision) combination not built */
  FFC_EBOUNDS = -6,       /* status word: an index (slot, dof, vertex) was out of range */
  FFC_ETIMEOUT = -7       /* status word: a bounded device wait gave up */
} ffc_status;

/* Forms of Section 3.3 of the paper, and the linear form L(v) = int v f dx of
 * Section 2.1 (the right-hand side of the Poisson specification in Section 5.5). */
typedef enum {
  FFC_MASS = 0,           /* int v u dx                         (test case 1) */
  FFC_POISSON = 1,        /* int grad v . grad u dx             (test case 2) */
  FFC_NS_CONVECTION = 2,  /* int v . (w . grad) u dx, w given   (test case 3) */
  FFC_ELASTICITY = 3,     /* int 2 mu eps(v):eps(u) + lambda div v div u dx (test case 4) */
  FFC_SOURCE = 4          /* int v f dx, f = sum_t f_t phi_t given per cell (rank 1):
                           * A0[i][t] = int_{K0} Psi_i Psi_t, G_K[t] = |det J| f_t */
} ffc_form_kind;

typedef enum { FFC_TRIANGLE = 2, FFC_TETRAHEDRON = 3 } ffc_cell; /* value = spatial dimension d */

/* Arithmetic of the contraction A0 : G. J, its cofactors (adjugate) and det J are always
 * FP64: that is where a near-degenerate cell cancels. For FFC_FP64 the inverse
 * K = adj(J) / det J and G_K are FP64. For FFC_FP32 and the tensor-core precisions G_K
 * is formed in FP32, the type it is rounded to anyway (the tensor cores further split it
 * into operand parts): the dense kernels form K in FP32 from the FP64 adjugate and
 * determinant (a well-conditioned step; cells with |det J| outside [1e-30, 1e30] divide
 * in FP64), the block algorithm takes an FP64 K. FP64 is the CSR accumulation type of
 * ffc_assemble. Tensor-core precisions are built for tetrahedra: convection P2,
 * elasticity P1-P3, Poisson P2-P4, mass P3-P4 (others, and every linear form, return
 * FFC_EUNSUPPORTED); for the quadrature representation see ffc_tabulate_quadrature. */
typedef enum {
  FFC_FP64 = 0,   /* FP64 contraction, A_K stored as double */
  FFC_FP32 = 1,   /* FP32 G and A0, FP32 accumulation on CUDA cores, A_K stored as float */
  FFC_TF32 = 2,   /* tcgen05 kind::tf32, one product, FP32 accumulation in TMEM, float out */
  FFC_TF32X3 = 3, /* tcgen05 kind::tf32 with hi/lo splits of G and A0 (three products), float out */
  FFC_BF16X3 = 4, /* tcgen05 kind::f16 (BF16) with three-part splits of G and A0 (six products), float out */
  FFC_FP64_OZAKI = 5 /* FP64 by exact products of 7-bit digits on tcgen05, double out (the quadrature calls only;
                        FFC_EINVAL elsewhere) */
} ffc_precision;

/* How the CUDA-core precisions (FFC_FP64, FFC_FP32) evaluate the vector forms.
 * DENSE contracts the full reference tensor A0 (|alpha| = 90 for convection P2, 81 for
 * elasticity); BLOCK uses the Cartesian-product structure of the component-blocked
 * vector basis (Section 3.5): the element tensor's n_s x n_s blocks are contractions
 * of a reduced reference tensor R[n_s*n_s][k] with per-cell reduced geometry blocks
 * (convection: one block of n_s*d entries on the diagonal; elasticity: nine blocks of
 * d*d), the same sums with 27x / 9x fewer multiply-adds. AUTO = BLOCK for the vector
 * forms, DENSE otherwise. The tensor-core precisions always contract densely. */
typedef enum { FFC_ALG_AUTO = 0, FFC_ALG_DENSE = 1, FFC_ALG_BLOCK = 2 } ffc_algorithm;

/* Device status bits returned by ffc_status_poll. */
#define FFC_FLAG_DEGENERATE 0x1u
#define FFC_FLAG_BOUNDS 0x2u
#define FFC_FLAG_TIMEOUT 0x4u

/*
 * ffc_form_create -- compile a form: build the reference tensor
 *   A0[i1*n + i2][alpha] = int_{K0} prod dPhi/dX dX        (Section 3.2, A0 equation)
 * once, in FP64, by collapsed Gauss-Jacobi quadrature on the reference simplex
 * (Section 5.3 and Section 6), exact for the integrand degree.
 *   form   ffc_form_kind; cell ffc_cell; degree q of the Lagrange space (1..4;
 *          the convection form takes 1..2, elasticity 1..3, vector forms need tets;
 *          the source form's coefficient f lives in the same space as v).
 *   mu, lambda  elasticity parameters (ignored by the other forms).
 *   out    receives a new handle; release with ffc_form_destroy.
 * Returns FFC_EINVAL / FFC_EUNSUPPORTED / FFC_ENOMEM. Host-only: no device memory
 * is touched until a launch needs the reference tensor on a device.
 */
int ffc_form_create(int form, int cell, int degree, double mu, double lambda, ffc_form** out);

/* n_local = n (local dofs per cell), n_alpha = |alpha| (entries of G_K),
 * n_coeff = per-cell coefficients the form reads (30 for vector-P2 convection, n for
 * the source form, else 0). */
int ffc_form_info(const ffc_form* f, int* n_local, int* n_alpha, int* n_coeff);

/* Rank of the form's tensor (Section 3.1): 2 for a bilinear form (element matrix),
 * 1 for a linear form (element vector). */
int ffc_form_rank(const ffc_form* f, int* rank);

/* Raw reference tensor (the "raw format" output of Section 5.4):
 * host_out double [n^rank][n_alpha], row-major. */
int ffc_form_reference_tensor(const ffc_form* f, double* host_out);

/* Selects the evaluation of the vector forms (ffc_algorithm); FFC_EINVAL otherwise. */
int ffc_form_set_algorithm(ffc_form* f, int algorithm);

/* Frees host data and any device copies of the reference tensor. NULL is ignored. */
void ffc_form_destroy(ffc_form* f);

/*
 * ffc_tabulate -- element tensors A^K = A0 : G_K for n_elem cells (Section 3.2,
 * eq. (tensorproduct); the per-cell evaluation the generated eval() of Section 5.5
 * performs).
 *   cells     device int32 [n_elem][d+1] vertex ids (local vertex order as given)
 *   vertices  device double [n_vert][d]
 *   coeffs    device double [n_elem][n_coeff] (convection: w on each cell, component
 *             blocked like the basis; source: f on each cell), NULL when n_coeff == 0
 *   A_K       device [n_elem][n][n] ([n_elem][n] for a linear form), double for
 *             FFC_FP64, float otherwise
 *   precision ffc_precision
 * n_elem == 0 launches nothing and returns FFC_OK. A vertex id outside
 * [0, n_vert) is replaced by 0 and sets FFC_FLAG_BOUNDS (never read out of range).
 * Callers holding per-cell (gathered) vertex coordinates [n_elem][d+1][d] pass them as
 * `vertices` with n_vert = n_elem*(d+1) and cells[e] = {(d+1)e, ..., (d+1)e+d}.
 */
int ffc_tabulate(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                 int64_t n_vert, const double* coeffs, void* A_K, int precision, void* stream);

/*
 * ffc_csr_pattern -- sparsity pattern of the assembled matrix (host, setup).
 * The pattern holds every (row, col) pair of dofs that share a cell (Algorithm 2
 * touches exactly those entries), columns sorted ascending within each row.
 *   dofmap  host int32 [n_elem][n_local], global ids in [0, n_dof)
 *   row_ptr host int64 [n_dof + 1] (always written)
 *   nnz     receives the number of stored entries
 *   col     host int32 [nnz] or NULL; written only when col_capacity >= nnz
 *   slot    host int32 [n_elem][n_local][n_local] or NULL: position in `col` of
 *           (dofmap[e][i1], dofmap[e][i2]); written together with col
 * Call once with col = NULL to learn nnz, then again with buffers.
 * Uses all host threads of the process affinity mask. FFC_EBOUNDS if a dof id
 * is out of range; FFC_EINVAL if nnz would exceed INT32_MAX (slots are int32).
 */
int ffc_csr_pattern(int64_t n_elem, int n_local, const int32_t* dofmap, int64_t n_dof,
                    int64_t* row_ptr, int64_t* nnz, int32_t* col, int64_t col_capacity, int32_t* slot);

/*
 * ffc_assemble -- Algorithm 2 fused on the device: for every cell compute A^K
 * (as ffc_tabulate, never written to memory) and add it into the CSR values,
 *   csr_val[slot[e][i1][i2]] += A^K[i1][i2]     (FP64 atomic adds).
 *   slot     device int32 [n_elem][n][n] from ffc_csr_pattern
 *   csr_val  device double [nnz], accumulated into (zero it first for a fresh matrix)
 * A linear form is added into a global vector the same way, b[slot[e][i]] += b^K[i]:
 * `slot` is then the dof map itself (device int32 [n_elem][n]), `csr_val` the vector
 * b and `nnz` its length (the number of global dofs).
 * Slots >= nnz are skipped and set FFC_FLAG_BOUNDS. Summation order of the atomic
 * adds is not deterministic (results agree to rounding).
 */
int ffc_assemble(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                 int64_t n_vert, const double* coeffs, const int32_t* slot, double* csr_val, int64_t nnz,
                 int precision, void* stream);

/*
 * ffc_assemble_pair -- ffc_assemble for two bilinear forms on the same space (same cell,
 * degree and dof map, hence the same CSR pattern and slots), e.g. the mass and stiffness
 * matrices of a time step or an eigenproblem:
 *   csr_val_a[slot[e][i1][i2]] += A_a^K[i1][i2],  csr_val_b[slot[e][i1][i2]] += A_b^K[i1][i2]
 * The pair (mass, Poisson), in either order, with FFC_FP32 runs as one launch: the cell's
 * geometry is computed once and each slot is loaded once for both matrices; each matrix
 * receives the contributions ffc_assemble computes for it (the same arithmetic; the sums
 * agree to rounding, the atomic order being free). Any other pair of forms without
 * coefficients runs as two ffc_assemble calls. csr_val_a and csr_val_b are distinct
 * device double [nnz] arrays, accumulated into. FFC_EINVAL for forms on different
 * spaces or one array passed twice; FFC_EUNSUPPORTED for forms with coefficients.
 */
int ffc_assemble_pair(const ffc_form* fa, const ffc_form* fb, int64_t n_elem, const int32_t* cells,
                      const double* vertices, int64_t n_vert, const int32_t* slot, double* csr_val_a,
                      double* csr_val_b, int64_t nnz, int precision, void* stream);

/*
 * ffc_scatter_add -- the insertion step of Algorithm 2 (Section 2.2) on its own: adds
 * precomputed element tensors into the CSR values,
 *   csr_val[slot[e][i]] += A_K[e][i]     for e < n_elem, i < n_entries (FP64 atomic adds).
 *   A_K        device [n_elem][n_entries], double (precision FFC_FP64) or float
 *              (FFC_FP32), e.g. from ffc_tabulate: n_entries = n*n, or n for a linear form
 *   slot       device int32 [n_elem][n_entries] from ffc_csr_pattern (the dof map for a
 *              linear form)
 *   csr_val    device double [nnz], accumulated into
 * ffc_assemble fuses this step into the contraction; this entry serves element tensors
 * computed elsewhere. Slots outside [0, nnz) are skipped and set FFC_FLAG_BOUNDS; the
 * order of the atomic adds is not deterministic.
 */
int ffc_scatter_add(int64_t n_elem, int n_entries, const void* A_K, int precision, const int32_t* slot,
                    double* csr_val, int64_t nnz, void* stream);

/*
 * ffc_tabulate_adjoint -- reverse mode of ffc_tabulate with respect to the vertex
 * coordinates (chain rule through G_K(J) of the Poisson form, Section 3.3 test
 * case 2, and J = [x_1 - x_0, ...]):
 *   dG[alpha]   = sum_i A0[i][alpha] * dA_K[e][i]
 *   dJ          from dG through G = |det J| K K^T, K = J^{-1}
 *   dvertices[cells[e][j]] += dJ contributions   (FP64 atomic adds)
 *   dA_K       device double [n_elem][n][n], the upstream gradient dL/dA_K
 *   dvertices  device double [n_vert][d], accumulated into
 * Poisson forms only (FFC_EUNSUPPORTED otherwise).
 */
int ffc_tabulate_adjoint(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                         int64_t n_vert, const double* dA_K, double* dvertices, void* stream);

/*
 * Batched heterogeneous assembly (Algorithm 2 over many independent problems in one
 * persistent launch). Each item is one (mesh, form) problem exactly as for
 * ffc_assemble (device pointers, caller-owned); the arithmetic is FP64 geometry,
 * FP32 contraction (FFC_FP32) and FP64 CSR accumulation. Forms carried: elasticity
 * P1-P3, Poisson P1-P2, mass P1, all on tetrahedra (others: FFC_EUNSUPPORTED).
 * The kernel takes tiles of cells from one global atomic counter; no CTA waits for
 * another. The library allocates a small work table per tile variant.
 */
typedef struct {
  const ffc_form* form;
  int64_t n_elem;
  const int32_t* cells;     /* device int32 [n_elem][4] */
  const double* vertices;   /* device double [n_vert][3] */
  int64_t n_vert;
  const double* coeffs;     /* device, or NULL (no batched form reads coefficients) */
  const int32_t* slot;      /* device int32 [n_elem][n][n] */
  double* csr_val;          /* device double [nnz] */
  int64_t nnz;
} ffc_batch_item;

/* zero_csr != 0: every run first zeroes each item's csr_val (a fresh assembly). */
int ffc_batch_create(const ffc_batch_item* items, int n_items, int zero_csr, ffc_batch** out);
/* Times the twelve tile variants (256 threads per block, or 416 with registers bounded for
 * one or for two resident blocks; x 16, 32, 64 or 128 cells per thread group and tile) on
 * the caller's data, keeps the fastest and returns it
 * (either output pointer may be NULL); leaves every csr_val zeroed. */
int ffc_batch_tune(ffc_batch* b, void* stream, int* cells_per_tile_group, int* threads_per_block);
/* One persistent launch (use_graph = 0), or the same work captured once into a CUDA
 * graph on `stream` and replayed (use_graph != 0). */
int ffc_batch_run(ffc_batch* b, int use_graph, void* stream);
int ffc_batch_info(const ffc_batch* b, int* n_items, long long* total_tiles, int* cells_per_tile_group,
                   int* threads_per_block);
void ffc_batch_destroy(ffc_batch* b);

/*
 * Row-owner assembly: Algorithm 2 (Section 2.2) with its loops ordered by global row.
 * Algorithm 2 adds the element tensor of each cell into the matrix; the entries of
 * global row r therefore receive exactly the element-tensor rows A^K[i1][:] of the
 * cells K with dofmap[K][i1] = r (the "pairs" (K, i1) of row r). The rows are cut into
 * chunks of consecutive rows (at most 4096 stored entries each); one CTA sums a chunk in
 * shared memory, computing the entries from a per-cell geometry tensor G_K
 * (A^K = A0 : G_K, Section 3.2), and writes the chunk's CSR values once, in order. No
 * global atomics, no zeroing: every CSR value is overwritten.
 *
 * The sums are in fixed point: each contribution (FP32 or FP64, as the contraction
 * produced it) is rounded to a grid with one unit per chunk and form, where 2^(eb-1)
 * bounds every partial sum of the chunk's entries (the largest per-pair bound
 * max|A0[i1][.][.]| * sum|G_K| times the most pairs of one row): u = 2^(eb-62) (63 bits,
 * three 21-bit digits) for FFC_FP64 and u = 2^(eb-31) (31 bits, one digit) for FFC_FP32.
 * The digits are summed as 32-bit integers in shared memory, so the sums do not depend on
 * their order, and each result is rounded once to FP64. Per entry: |result - exact sum
 * of the contributions| <= m * u / 2 + ulp(result) with m the entry's number of
 * contributions (u / 2 < 2^-30 B for FP32, 2^-61 B for FP64, B the chunk's bound): for
 * FP32 well inside 1e-6 of the row's sum of |contributions|. Results are bitwise
 * reproducible.
 *
 * ffc_row_plan_create -- the row view of a dof map and its CSR pattern, built on the
 * device once per (mesh, space):
 *   dofmap   device int32 [n_elem][n_local], global ids in [0, n_dof), n_local <= 64
 *   row_ptr  device int64 [n_dof + 1], col device int32 [nnz]: the pattern of
 *            ffc_csr_pattern (columns sorted within each row), copied to the device
 * The plan stores, per chunk, the chunk's pairs grouped by local index i1 as
 * e * n_local + i1, the work units (pieces of one group), and for every pair and local
 * column i2 the position of column dofmap[e][i2] inside the chunk (uint16). It owns
 * about n_elem * n_local * (2 * n_local + 4) + n_dof * 8 bytes of device memory plus an
 * [n_elem][12]-double geometry scratch (ffc_row_plan_layout reports the exact figure);
 * row_ptr is copied, so dofmap, row_ptr and col may be freed afterwards. The call
 * synchronises `stream`.
 * Errors: FFC_EBOUNDS for a dof id outside [0, n_dof) or a (row, col) pair of a cell
 * missing from the pattern; FFC_EINVAL for n_local outside [2, 64], a row with more than
 * 4096 entries or more than 320 pairs (a dof shared by more than 320 cells), a row_ptr
 * that is not monotone within [0, nnz], or n_elem * n_local >= 2^31.
 */
int ffc_row_plan_create(int64_t n_elem, int n_local, const int32_t* dofmap, int64_t n_dof, const int64_t* row_ptr,
                        const int32_t* col, int64_t nnz, void* stream, ffc_row_plan** out);
/* Rows, stored entries, longest row and most cells sharing one dof. */
int ffc_row_plan_info(const ffc_row_plan* p, int64_t* n_dof, int64_t* nnz, int* max_row, int* max_incidence);
/* Chunks, entries and pairs of the largest chunk, bytes of the largest chunk's plan data
 * (work units, pairs and positions) and the plan's device memory in bytes. Any output
 * pointer may be NULL. */
int ffc_row_plan_layout(const ffc_row_plan* p, int64_t* n_chunks, int* max_chunk_values, int* max_chunk_pairs,
                        int* max_region_bytes, int64_t* device_bytes);
void ffc_row_plan_destroy(ffc_row_plan* p);

/*
 * ffc_assemble_rows -- the assembled matrix of a mass or Poisson form (any degree,
 * triangles and tetrahedra) by row-owner assembly with `plan`:
 *   csr_val[k] = sum of A^K[i1][i2] over the cells and local pairs that map to entry k,
 * for every k < nnz (overwritten). cells / vertices / n_vert as for ffc_tabulate, for
 * the cells the plan was built from. precision FFC_FP32: G_K and the contraction in
 * FP32 exactly as ffc_assemble computes them (the same contributions), FFC_FP64: in FP64.
 * Two launches on `stream`: the geometry tensors into the plan's scratch, then the rows.
 * Calls that share a plan must be ordered on one stream (they share the scratch).
 * A non-finite G_K (a degenerate cell, FFC_FLAG_DEGENERATE) makes the values of the
 * chunk that holds its rows NaN. Other forms: FFC_EUNSUPPORTED. The plan's n_local must
 * equal the form's.
 */
int ffc_assemble_rows(const ffc_form* f, const ffc_row_plan* plan, const int32_t* cells, const double* vertices,
                      int64_t n_vert, double* csr_val, int precision, void* stream);

/*
 * ffc_assemble_rows_pair -- ffc_assemble_rows for two forms on the plan's space into two
 * matrices with the plan's pattern. The pair (mass, Poisson), in either order, is one
 * pass: each cell's geometry is computed once, each position is read once and feeds both
 * matrices; every value equals the one ffc_assemble_rows writes for that form, bit for
 * bit. Two forms of one kind run as two ffc_assemble_rows calls. csr_val_a and csr_val_b
 * are distinct device double [nnz] arrays, overwritten.
 */
int ffc_assemble_rows_pair(const ffc_form* fa, const ffc_form* fb, const ffc_row_plan* plan, const int32_t* cells,
                           const double* vertices, int64_t n_vert, double* csr_val_a, double* csr_val_b,
                           int precision, void* stream);

/*
 * Quadrature as a tensor contraction (Section 3.4, "Curvilinear elements"). When the map
 * F_K from the reference simplex K0 is not affine, the Jacobian cannot be taken out of
 * the integral; replacing the integral by a quadrature sum over points X_k with weights
 * w_k keeps the element tensor a contraction, with one extra index for the points:
 *   A^K_{i1 i2} ~= sum_k w_k integrand(X_k) |det F_K'(X_k)| = A~0[i][j] G~_K[j],
 *   j = k * n_g + g over the points k and the per-point geometry entries g:
 *   mass     n_g = 1:          A~0[i][k]     = w_k Phi_i1(X_k) Phi_i2(X_k)
 *                              G~_K[k]       = |det F_K'(X_k)|
 *   Poisson  n_g = d(d+1)/2:   A~0[i][(k,g)] = w_k (dPhi_i1/dX_a dPhi_i2/dX_b + [a != b]
 *                                              dPhi_i1/dX_b dPhi_i2/dX_a)(X_k)
 *                              G~_K[(k,g)]   = |det F_K'(X_k)| (F'^-1 F'^-T)[a][b](X_k)
 *   for the pairs g = (a <= b), diagonal pairs first, then (0,1) [, (0,2), (1,2)].
 * A~0 is computed once per form on the host (FP64); G~_K per cell on the device. The map
 * is the geometry interpolant of degree `geometry_degree` (1: affine, 2: quadratic),
 * F_K(X) = sum_n x_n Psi_n(X) over the cell's geometry nodes x_n in the local dof order
 * of the P_g Lagrange space. The rule is the collapsed Gauss-Jacobi rule of
 * Karniadakis & Sherwin exact for polynomial degree `quad_degree` (the rule A0 uses):
 * m = ceil((quad_degree + 1) / 2) points per direction, direction k weighted by
 * (1 - u)^k, X_k = u_k prod_{l > k} (1 - u_l). On affine cells with quad_degree at least
 * the integrand's degree the result equals ffc_tabulate's to rounding.
 *
 * ffc_qform_create -- form FFC_MASS or FFC_POISSON, cell FFC_TRIANGLE / FFC_TETRAHEDRON,
 * degree 1..4, geometry_degree 1 or 2, quad_degree 0..20. FFC_EINVAL otherwise.
 * ffc_qform_info -- local dofs n, geometry nodes per cell, quadrature points, and the
 * contraction length K = points * n_g.
 * ffc_qform_reference_tensor -- A~0 as [n * n][K] doubles (j = k * n_g + g).
 * ffc_qform_rule -- the points [N][d] (reference coordinates) and weights [N] (summing
 * to 1/d!); either pointer may be NULL.
 */
int ffc_qform_create(int form, int cell, int degree, int geometry_degree, int quad_degree, ffc_qform** out);
int ffc_qform_info(const ffc_qform* f, int* n_local, int* n_geometry, int* n_points, int* k_contract);
int ffc_qform_reference_tensor(const ffc_qform* f, double* out);
int ffc_qform_rule(const ffc_qform* f, double* points, double* weights);
void ffc_qform_destroy(ffc_qform* f);

/*
 * ffc_tabulate_quadrature -- A_K = A~0 : G~_K for a batch of cells:
 *   cells   device int32 [n_elem][n_geometry], geometry node ids in [0, n_nodes)
 *   nodes   device double [n_nodes][d], node coordinates
 *   A_K     device [n_elem][n][n], double (FFC_FP64, FFC_FP64_OZAKI) or float (the others),
 *           16-byte aligned
 * FFC_FP64: G~_K and the contraction in FP64. FFC_FP32: F', its determinant and inverse
 * in FP64, G~_K rounded to FP32, the contraction in FP32. A node id out of range sets
 * FFC_FLAG_BOUNDS (its cell's tensor is then computed from node 0); a point where
 * |det F'| <= 1e-14 h^d (h the largest node distance from node 0) sets
 * FFC_FLAG_DEGENERATE.
 * FFC_TF32 / FFC_TF32X3 / FFC_BF16X3 (element tensors of at most 512 entries, up to four
 * 128-entry M tiles: P1-P3 on tets, P1-P4 on triangles, else FFC_EUNSUPPORTED): the
 * contraction on the tensor cores (tcgen05) in 128-cell tiles, A~0 split into TF32 or
 * BF16 parts on the host, G~_K per point in FP32 split the same way on the device, the
 * tensor cores accumulating G~_K(X_k) - G~_K(centroid) and the centroid term added in
 * FP32, A_K written as float. The split precisions keep FP32 accuracy; FFC_TF32 alone has
 * TF32's 11-bit precision (times the deviations' relative size).
 * FFC_FP64_OZAKI (element tensors of at most 128 entries, and K = points x n_g
 * at most 400, else FFC_EUNSUPPORTED): A_K as double, FP64-accurate, with the contraction
 * on the tensor cores by exact products of small-integer digits (the splitting of Ozaki,
 * Ogita, Oishi and Rump, Numer. Algorithms 59, 2012): each row of A~0 and each cell's
 * column of G~ (computed in FP64) scaled by a power of two and written as eight balanced
 * 7-bit digits, exact in BF16; the digit products summed per digit order in FP32 TMEM
 * accumulators, exact integers for K <= 400; recombined in 64-bit integers and rounded
 * once to FP64. Truncation below 2^-56 of the row and column scales. A value beyond a
 * column's scale (a cell whose FP32 and FP64 geometry disagree, a NaN) is clamped and
 * sets FFC_FLAG_DEGENERATE.
 * FFC_EINVAL for other precisions or bad pointers.
 *
 * ffc_assemble_quadrature -- Algorithm 2 fused, as ffc_assemble:
 *   csr_val[slot[e][i1][i2]] += A_K[e][i1][i2]   (FP64 atomic adds)
 * with slot from ffc_csr_pattern of the P_degree dof map (the geometry nodes are only an
 * input of the map, not of the pattern); the precisions and limits of
 * ffc_tabulate_quadrature (the tensor-core kernels add in their drain). slot (device
 * int32 [n_elem][n][n]) and csr_val (device double [nnz]) must be naturally aligned and
 * nnz > 0 (FFC_EINVAL otherwise); a slot outside [0, nnz) is skipped and sets
 * FFC_FLAG_BOUNDS.
 */
int ffc_tabulate_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                            int64_t n_nodes, void* A_K, int precision, void* stream);
int ffc_assemble_quadrature(const ffc_qform* f, int64_t n_elem, const int32_t* cells, const double* nodes,
                            int64_t n_nodes, const int32_t* slot, double* csr_val, int64_t nnz, int precision,
                            void* stream);

/*
 * ffc_status_poll -- return the device status bits (FFC_FLAG_*) accumulated by earlier
 * launches on the current device, and clear them. The read and the clear are ordered on
 * `stream`, and the call then waits for `stream` only: launches on other streams keep
 * running, and bits they set after the read are reported by a later poll.
 */
int ffc_status_poll(void* stream, uint32_t* flags);

/*
 * ffc_tabulate_static -- ffc_tabulate for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment variant of ffc_tabulate.
 *
 * Frameworks that route every device allocation through their own pool, and
 * applications that fix their device memory before loading this library, cannot
 * let the library call cudaMalloc. This entry point allocates nothing: the
 * reference tensor and the status word live in one fixed 2 MiB (+256 B) device
 * array compiled into the library, which every GPU that loads the library holds
 * until the process exits. The caller passes inputs and outputs as for ffc_tabulate.
 *   precision   FFC_FP64 or FFC_FP32 only
 *   host_flags  NULL, or receives the FFC_FLAG_* bits of this call; when non-NULL
 *               the call synchronises `stream` before returning
 * Forms whose reference tensor does not fit (4 copies of n*n*|alpha| values plus the
 * reduced tensor of the block algorithm, e.g. elasticity P3) are rejected with FFC_EINVAL
 * before any device work. The kernels are those ffc_tabulate chooses (the vector forms
 * follow ffc_form_set_algorithm), so the results equal ffc_tabulate's bit for bit.
 * The first call on a device looks up the array's device address (with that device
 * current). The reference tensor is uploaded from the form's host copy on every call,
 * so the call returns FFC_EINVAL while `stream` is being captured into a graph. All
 * calls share the array and leave their contents in it: each call clears the status
 * word and rewrites the reference tensor, so calls that overlap on the GPU race and must
 * be serialised by the caller.
 */
int ffc_tabulate_static(const ffc_form* f, int64_t n_elem, const int32_t* cells, const double* vertices,
                        int64_t n_vert, const double* coeffs, void* A_K, int precision, void* stream,
                        uint32_t* host_flags);

/*
 * ffc_diag_bounded_wait -- a check of the failure detection. Every device-side wait of the
 * library (the mbarrier waits between the warp roles of the tensor-core kernels) is
 * bounded: after its limit it gives up, sets FFC_FLAG_TIMEOUT and lets the kernel return,
 * so a stalled partner never hangs the GPU. This launches one CTA that waits, with that
 * same bounded wait and a limit of `polls` tries (at most 2^20), on an mbarrier that
 * nothing arrives at. Afterwards ffc_status_poll reports FFC_FLAG_TIMEOUT and the device
 * stays usable. FFC_EINVAL for polls > 2^20.
 */
int ffc_diag_bounded_wait(uint32_t polls, void* stream);

/*
 * ffc_diag_peak -- measures one compute ceiling of the current device (the denominators
 * of the roofline fractions of ALU-, tensor- and shared-atomic-bound kernels):
 *   FFC_PEAK_FP64_FMA, FFC_PEAK_FP32_FMA   fused multiply-add rate of the CUDA cores
 *                                          (flop/s, an FMA counts 2): eight independent
 *                                          chains per thread, 1024 threads per SM;
 *   FFC_PEAK_TF32_MMA, FFC_PEAK_BF16_MMA   dense tcgen05.mma rate (flop/s): one CTA per SM
 *                                          issuing M=128, N=256 MMAs (K = 8 tf32 / 16 bf16)
 *                                          on shared-memory operands, FP32 accumulation;
 *   FFC_PEAK_SMEM_ATOMIC_U32               32-bit shared-memory atomic adds per second,
 *                                          conflict-free addresses.
 * The probe is launched once to warm up and once timed with CUDA events on `stream`;
 * the call synchronises `stream`. rate receives the operations per second, seconds (may
 * be NULL) the timed launch's duration. FFC_ETIMEOUT if the tensor-core probe's bounded
 * wait gave up. There is no INT8 probe: sm_103a has no tcgen05 kind::i8.
 */
#define FFC_PEAK_FP64_FMA 0
#define FFC_PEAK_FP32_FMA 1
#define FFC_PEAK_TF32_MMA 2
#define FFC_PEAK_BF16_MMA 3
#define FFC_PEAK_SMEM_ATOMIC_U32 4
int ffc_diag_peak(int kind, double* rate, double* seconds, void* stream);

/* Human-readable name of a status code (static string). */
const char* ffc_status_string(int status);

/* Text of the last FFC_ECUDA / validation failure on this host thread (static per thread). */
const char* ffc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FFC_GB300_H */
