// Internal declarations of the bidomain library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bid.h"

namespace bid {

// ---------------------------------------------------------------- errors
int set_error(int code, const char* fmt, ...);
#define BID_CUDA_TRY(expr)                                                         \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess)                                                     \
            return ::bid::set_error(BID_ECUDA, "%s failed: %s (%s:%d)", #expr,     \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);   \
    } while (0)
#define BID_TRY(expr)                      \
    do {                                   \
        int rc_ = (expr);                  \
        if (rc_ != BID_OK) return rc_;     \
    } while (0)

// Count of kernel launches issued by this library (bid_kernel_launches).
void count_launches(int n);

// ---------------------------------------------------------------- host sparse
struct CsrHost {
    int64_t n = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
    int64_t nnz() const { return ptr.empty() ? 0 : ptr.back(); }
};

// Sliced ELLPACK with 32-row slices: element k of row r = 32*s + l lives at
// sptr[s] + 32*k + l (column-major inside a slice, so a warp reads a slice
// coalesced).  Padding entries have value 0 and column = the row itself.
struct SellDev {
    int32_t n = 0;
    int32_t nslices = 0;
    int32_t* sptr = nullptr;   // nslices + 1 offsets (elements)
    int32_t* col = nullptr;
    double* val = nullptr;
    int64_t stored = 0;        // stored entries including padding
};

// Upload a CSR matrix as sliced ELLPACK (32-row slices) / free it.  Padding
// entries read column = their row, or column 0 for rows at or beyond ncols
// (rectangular matrices with fewer columns than rows; ncols < 0: square).
int upload_sell(const CsrHost& A, SellDev* d, int64_t ncols = -1);
void free_sell(SellDev* d);

// ---------------------------------------------------------------- assembly
struct AssembledHost {
    int dim = 0;
    int64_t N = 0, NH = 0;
    std::vector<int64_t> perm;     // library index -> mesh node
    std::vector<double> coords;    // library order, N * dim
    CsrHost S1, Si, Sm;            // Sm: sigma_m stiffness on the heart (Sec. 5.2)
    std::vector<double> m, mH;     // lumped mass diagonals
};
int assemble_host(const bid_mesh* mesh, const bid_params* p, AssembledHost* out);

// ---------------------------------------------------------------- H-factor
#ifdef __CUDACC__
#define BID_HD __host__ __device__ __forceinline__
#else
#define BID_HD inline
#endif

// Factor of an SPD matrix A (n x n) in nested-dissection supernodal form.  For
// cluster s with pivot set I_s (ni entries, contiguous in the elimination
// order from `first`) and boundary set B_s (nb ancestor entries), the stored
// block is M_s = [L_ss^-1 ; L_Bs L_ss^-1], (ni + nb) x ni.  Its "dense rows"
// (the ni rows of L_ss^-1 and the boundary rows not in a low-rank group, nd in
// all) are stored packed, lower-trapezoidal and column-major: column j holds
// dense rows q = j .. nd-1, contiguous.  A low-rank group replaces m boundary
// rows by U (m x k, row-major) times V^T (V: ni x k, row-major).
struct HSnode {
    int32_t first, ni, nb, nd;
    int32_t bidx_off;   // B_s entries (vector indices) at bidx[bidx_off ...]
    int32_t u_off;      // uout[u_off + j]: slot of update row j in the parent's inputs
    int32_t inc_off;    // slot_stride input slots per frontal row at inb[inc_off + stride f + k]
                        // (child k's contribution), valid iff inc[...] >= 0
    int32_t height;
    int64_t data_off;   // packed dense columns
    int32_t drow_off;   // M_s row index of dense boundary row q (q >= ni) at drows[drow_off + q - ni]
    int32_t lr_begin, lr_end;
    int32_t large;      // 1: chunked upper-level tasks (may hold low-rank groups); 0: flat items
    int32_t v_off;      // large clusters: backward input staged at vbuf[v_off ...]
    int32_t nchild;     // children in the cluster tree (0: no incoming updates; up to 4 for a
                        // cluster merged with its two children's separators)
};
// Update slots per frontal row of a cluster: one per child, two or four.
BID_HD int slot_stride(const HSnode& s) { return s.nchild > 2 ? 4 : 2; }
constexpr int MAX_CHILDREN = 4;
// Number of stored (nonzero) entries of columns 0 .. j-1 of the dense part.
BID_HD int64_t col_offset(int64_t nd, int64_t j) { return j * nd - j * (j - 1) / 2; }
// Start of column j inside the cluster's dense data.  Column c holds rows
// c .. nd-1 followed by p_c zeros, p_c = (1 - (nd - c)) mod vec, so that
// start(j) - j is a multiple of vec: row q of every column then sits at an
// address congruent to q modulo vec, and a thread can read rows q .. q+vec-1
// (q a multiple of vec) of any column as one aligned 16-byte vector.
BID_HD int64_t col_start(int64_t nd, int64_t j, int64_t vec) {
    const int64_t r0 = ((1 - nd) % vec + vec) % vec;
    const int64_t m = j % vec;
    const int64_t wrap = m - (vec - r0);
    const int64_t pad = (j / vec) * (vec * (vec - 1) / 2) + m * r0 + m * (m - 1) / 2 -
                        vec * (wrap > 0 ? wrap : 0);
    return col_offset(nd, j) + pad;
}

struct HLr {
    int32_t s, row0, m, k;      // rows [row0, row0+m) of M_s (boundary rows)
    int64_t off_u, off_v;
    int32_t t_off, pad;         // slot of V^T w (forward) / U^T v (backward) in tbuf
};
// Positions (elimination order), the boundary lists bidx / uout and the
// update slots are all numbered in the data order described below.
// Flat work of the small clusters of one level.  The small clusters of a
// level are cut into groups of consecutive clusters whose packed data is
// contiguous in `data` (a group's factor bytes are [dstart, dstart + nbytes)
// in elements / bytes, 16-byte aligned); one CTA per group copies them into
// shared memory with one bulk copy, stages the inputs and then computes:
//  forward:  one unit per aligned row group (vec rows) of a cluster, over all
//            its columns (uf units per group);
//  backward: one unit per column of a cluster, over all its rows (ub units).
// The update slots of a group's clusters are contiguous too (slots are
// numbered in the same order as the data), and copied by a second bulk copy
// when some cluster of the group has children.  Slots that no child writes
// stay zero (each factor owns its zero-initialised slot array), so the flat
// kernels add both slots of a frontal row without validity checks.
// A group holds at most STAGE_CL clusters, STAGE_MAX staged values in either
// pass and, unless it is a single cluster, HBuildOpts::group_bytes bytes of
// data: small CTAs (FLAT_THREADS threads, the group's data, slots,
// descriptors and staged inputs in dynamic shared memory sized per level) so
// that many groups are resident per SM and their load phases overlap.
struct FGroup {
    int64_t dstart;                 // element offset of the group's data
    int64_t sstart;                 // first update slot of the group's clusters
    int32_t nbytes;                 // data bytes copied (multiple of 16)
    int32_t sbytes;                 // update-slot bytes copied (0: no cluster has children)
    int32_t c0, c1;                 // clusters gcl[c0 .. c1)
    int32_t wf, wb;                 // staged values, forward / backward
    int32_t uf, ub;                 // units, forward / backward
    int32_t pstart;                 // first pivot position (the group's pivots: wf positions)
    int32_t bstart, nbt;            // its boundary rows: bidx / uout [bstart, bstart + nbt)
    int32_t pad;
};
struct GCl {                        // a cluster of a group: descriptor and prefixes
    int32_t first, ni, nd, doff;    // doff: data offset inside the group (elements)
    int32_t soff, boff, nchild, s;      // slot / boundary-row offsets inside the group; cluster
    int32_t woff_f, woff_b, uf0, ub0;   // woff_f = uf... pivot offset inside the group
};
// Work item of a large-cluster kernel.
//  upper forward:   s >= 0: dense rows [a0, a1) x columns [b0, b1); when the
//                   row chunk is split over nparts column chunks, partial sums
//                   go to pbuf[part + c*(a1-a0) + row] and the last CTA of
//                   ticket `ticket` finishes the rows;  s < 0: low-rank group
//                   g = -1 - s, rows [a0, a1) of the group
//  upper backward:  cluster s, columns [a0, a1), b0 warps per column
struct HTask {
    int32_t s, a0, a1, b0, b1, part, ticket, nparts;
};
// A large cluster whose whole block (its low-rank groups' U and V, then its
// dense columns) fits one CTA's shared memory.  Such a cluster has no tasks:
// one CTA per cluster and pass (k_mid_fwd / k_mid_bwd) copies the block with
// bulk copies, stages its inputs and computes every row (forward) or column
// (backward), the low-rank products included, with the partial sums of a row
// or column combined in shared memory in a fixed order.  Its low-rank groups
// follow the task clusters' groups of the same level (HFactorHost::ulr_mid),
// so the backward preparation launch covers only the task clusters.
struct MidCl {
    int64_t blk;        // element offset of the block in `data` (16-byte aligned)
    int32_t s;          // the cluster
    int32_t nbytes;     // bytes copied: the block and two trailing vectors (multiple of 16)
    int32_t dense;      // element offset of the dense columns inside the block
    int32_t npair;      // sum of the ranks of its low-rank groups
    int32_t ng;         // its low-rank groups
    int32_t pad;
};
// Dynamic shared memory of a mid launch, per level (byte offsets): the block
// at 0, then w (forward input / backward dense-row input, nd + vec values),
// ib (forward: incoming updates of the boundary rows, FP64; backward: -x_B),
// red (partial sums), tl / tp (low-rank products and their partial sums),
// gd (group descriptors), pt (one MidPair per low-rank product entry),
// bi (forward: the boundary rows' update slots; backward: their vector
// indices), dr (dense boundary rows, minus ni), po (backward: the pivots'
// vector indices).
struct MidLayout {
    int32_t w, ib, red, tl, tp, gd, pt, bi, dr, po, total;
    int32_t pa, tq, ad, pad;   // wide clusters: row partials, product partials, WideAdj table
};
struct MidPair {    // entry l of the low-rank group holding product entry p
    int32_t voff, uoff, k, rb;   // V(0, l), U(0, l) inside the block; rank; first row - ni
    int32_t m, pad0, pad1, pad2;
};
// A large cluster too big for one CTA but within WIDE_MAX_CTAS CTAs' shared
// memory ("wide"): one thread-block cluster of C CTAs per tree cluster and
// pass (k_wide_fwd / k_wide_bwd).  CTA c holds a column slice [j0, j1) of
// the dense block and the same rows of every low-rank V, plus the whole U of
// the groups it owns, each piece bulk-copied into its shared memory.  Forward:
// every CTA forms the partial sums of the dense rows and of t = V^T w over its
// columns; after a cluster barrier, CTA c sums the C partials of its rows
// [q0, q1) and of its groups' t (distributed shared memory, rank order) and
// writes y, the update slots and its groups' low-rank rows.  Backward: each
// CTA computes its groups' t = U^T v; after a cluster barrier every CTA reads
// all t from their owners and computes its columns.  A wide cluster keeps its
// chunked tasks as well: a level runs the wide kernels when all its large
// clusters are wide and the device can co-schedule the level's cluster size.
struct WideCl {
    int64_t blk;        // block start (elements)
    int32_t s;          // the tree cluster
    int32_t slice0;     // its slices: wslice[slice0 .. slice0 + C of the level)
};
struct WideSlice {      // one CTA of a wide cluster
    int32_t j0, j1;     // dense columns (j0 a multiple of vec)
    int32_t q0, q1;     // dense rows it finishes (forward)
    int32_t piece0, npiece;   // its bulk copies: wpiece[piece0 ..)
    int32_t nbytes;     // shared-memory bytes of its pieces
    int32_t adj0;       // per low-rank group of the cluster: wadj[adj0 + g]
    int64_t dbase;      // shared-memory element of dense entry (q, j) = dbase + col_start(j) - j + q
};
struct WidePiece {      // a bulk copy of elements [src, src + bytes / esz) to shared byte dst
    int64_t src;
    int32_t dst, bytes;
};
struct WideAdj {        // shared-memory element of V(j, l) = vadj + j k + l; of U(i, l) = uadj + i k + l
    int32_t vadj, uadj; // uadj < 0: the group's U is held by CTA `owner`
    int32_t owner, pad;
};
constexpr int WIDE_MAX_CTAS = 16;
constexpr int GRAM_NI_MIN = 128, GRAM_NI_MAX = 4096;    // root sizes that take the Gram product
constexpr int TOP_N_MAX = 2560;   // largest top block with the children (its dense G grows as n^2: 4097 rows
                                  // of the 2049^2 slice read 4x the bytes of the blocks they replace)
constexpr int GRAM_ROWS = 16;                           // rows of G per CTA (one per warp)
constexpr int WIDE_ND = 4096, WIDE_NB = 4096;   // largest dense rows / boundary rows
constexpr int WIDE_DATA_MAX = 160 * 1024;   // factor bytes of one CTA of a wide cluster
constexpr int MID_BYTES_DEFAULT = 96 * 1024;   // largest block of a mid cluster (bytes)
constexpr int MID_THREADS = 512;
constexpr int MID_NI = 256, MID_NB = 1024, MID_ND = 512, MID_PAIRS = 256, MID_GROUPS = 32;
constexpr int MID_SMEM_MAX = 224 * 1024;

struct HFactorHost {
    int64_t n = 0;
    int32_t pin = -1;                  // vector index fixed to zero, or -1
    std::vector<uint8_t> pinflag;      // several pinned indices (block-diagonal systems)
    int32_t height = 0;
    std::vector<int32_t> pidx;         // elimination position -> vector index
    std::vector<HSnode> sn;
    std::vector<int32_t> bidx, inc, drows, uout;
    std::vector<HLr> lr;
    std::vector<double> data;
    // small clusters: groups per level
    std::vector<FGroup> fg;
    std::vector<GCl> gcl;
    std::vector<int32_t> fg_ptr;               // level -> group range
    std::vector<int32_t> fg_bytes;             // level -> largest group data + slots (bytes)
    std::vector<int32_t> fg_nc, fg_wf, fg_wb;  // level -> most clusters / staged values of a group
    // large clusters, per level
    std::vector<int32_t> ulr_ptr;              // level -> low-rank groups [ptr, ptr+1)
    std::vector<int32_t> vg_ptr, vgl;          // level -> large clusters (backward staging)
    std::vector<int32_t> uf_ptr, ub_ptr;       // level -> task ranges
    std::vector<HTask> uft, ubt;
    std::vector<int32_t> u_ni_max, u_nd_max;   // level -> max ni / nd (shared memory)
    std::vector<int32_t> ulr_mid;              // level -> first low-rank group of its mid clusters
    std::vector<MidCl> mid;                    // mid clusters, level by level
    std::vector<int32_t> mid_ptr;              // level -> mid cluster range
    std::vector<WideCl> wide;                  // wide clusters, level by level
    std::vector<int32_t> wide_ptr;             // level -> wide cluster range
    std::vector<int32_t> wide_c;               // level -> CTAs per wide cluster (0: none)
    std::vector<WideSlice> wslice;
    std::vector<WidePiece> wpiece;
    std::vector<WideAdj> wadj;
    int64_t ubuf = 0, tbuf = 0, pbuf = 0, nslots = 0, vbuf = 0;
    int32_t ntickets = 0;
    int32_t vec = 2;
    int32_t lev_upper = 0;     // levels >= lev_upper hold only large clusters
    int64_t dense_entries = 0, lowrank_entries = 0;   // algorithmic (no padding)
    // Top-block Gram matrix.  When the top level holds one large cluster r with
    // no boundary and no low-rank groups, the forward and backward passes of the
    // top block -- r, and its children when the level below holds exactly them
    // -- are x_top = M_top^T (M_top w_top) with nothing in between, M_top =
    // L_top^-1 the inverse of the block's Cholesky factor (children's pivots,
    // then r's): G = M_top^T M_top (n_top x n_top, row-major, FP64) replaces
    // them by one product x_top = G w_top.  w_top of a top row is its xp entry
    // plus the update slots listed for it: a child's pivot, its own frontal row;
    // a pivot of r, the children's frontal boundary rows holding that node.
    int32_t gram_s = -1;                       // the root cluster, or -1
    int32_t gram_lev = -1;                     // the lowest level of the block
    std::vector<double> gram;
    std::vector<int32_t> top_cl;               // the block's clusters
    std::vector<int32_t> top_pos;              // per top row: its elimination position
    std::vector<int32_t> top_sptr, top_slot;   // per top row: slot pairs at top_slot[sptr[t] .. sptr[t+1])
    int64_t nsmall = 0, nlarge = 0, nlr = 0;
};

constexpr int GROUP_BYTES_DEFAULT = 12288;
struct HBuildOpts {
    double eps = 0.0;
    int leaf = 16;
    int block = 64;
    int threads = 0;
    int vec = 2;        // elements per 16-byte vector of the storage precision
    // Block-diagonal matrices (several independent problems): rows
    // [group_ptr[g], group_ptr[g+1]) form block g, which gets a cluster tree
    // of its own (leaf size group_leaf[g], or `leaf`); the factor is a forest.
    std::vector<int64_t> group_ptr;
    std::vector<int32_t> group_leaf;
    // Vector index of matrix row i in the vectors the solve reads and writes
    // (vmap[i] < vn); empty: the identity.
    std::vector<int32_t> vmap;
    int64_t vn = 0;
    // route every cluster from the lowest level holding a large cluster
    // upwards to the large-cluster kernels (needed by the persistent
    // upper-level path)
    bool upper_levels = false;
    int group_bytes = GROUP_BYTES_DEFAULT;   // factor bytes of a flat group (see FGroup)
    int group_bytes_leaf = 0;                // the same for the leaf level (0: group_bytes)
    int up_brows = 512;                      // target rows per warp of a large-cluster backward task
    int mid_bytes = MID_BYTES_DEFAULT;       // largest block of a mid cluster (MidCl); 0: none
    int wide_bytes = WIDE_DATA_MAX;          // factor bytes per CTA of a wide cluster (WideCl); 0: none
    // merge pass over the cluster tree (merge_upper_levels): subtrees of at
    // least merge_min nodes have their levels merged in pairs; 0: off
    int64_t merge_min = 0;
    // fronts with at least gpu_front_nf rows factorised on the GPU (gpu_front_factor)
    bool root_gram = true;                   // G = M^T M of the root (HFactorHost::gram) when it applies
    bool gpu_front = false;
    int gpu_front_nf = 1024;
};
// Dense numeric work of one front on the GPU (FP64): F (nf x nf, row-major,
// lower part used) -> M = [L_ss^-1 ; L_Bs L_ss^-1] (nf x ni, row-major) and
// the update matrix U = F_BB - L_Bs L_Bs^T (nb x nb, row-major, lower part
// meaningful), nb = nf - ni.  *bad: 0, or 1 + the index of a non-positive
// pivot.  One front at a time per process (serialised).
int gpu_front_factor(int nf, int ni, const double* F, double* M, double* U, int* bad);
// G = A A^T for A n x n (row-major, FP64) on the GPU (the tiled product kernel).
int gpu_gram_nt(int n, const double* A, double* G);
// A: symmetric CSR (full pattern).  coords: dim values per row (geometry of
// the unknowns, used by the nested dissection).  Every index in `pins` has its
// row and column replaced by the identity and its input entry set to zero
// (pseudo-inverse of a singular Neumann matrix, one pin per component).
int build_hfactor(const CsrHost& A, const double* coords, int dim,
                  const std::vector<int32_t>& pins, const HBuildOpts& o, HFactorHost* F);

// Limits shared by the build and the kernels.
constexpr int SMALL_NI = 64;     // a cluster is small when ni <= SMALL_NI and
constexpr int SMALL_NF = 320;    // ni + nb <= SMALL_NF (before compression)
constexpr int STAGE_MAX = 2048;  // staged input values of a flat CTA
constexpr int STAGE_CL = 64;     // clusters of a flat group
constexpr int FLAT_THREADS = 128;    // threads of a flat CTA
constexpr int UP_GROUPS = 64;    // row groups (of vec rows) of an upper forward task
constexpr int UP_SPLIT = 4;      // column splits of an upper forward task (16 columns each)
constexpr int UP_COLS = 64;      // columns of an upper forward task
constexpr int UP_THREADS = 256;  // threads of a low-rank group task (one per row)
constexpr int LR_ROWS = 256;     // max rows of a low-rank group
constexpr int LR_KMAX = 64;      // largest rank kept in a low-rank group

// ---------------------------------------------------------------- device factor
struct HFactorDev {
    int64_t n = 0;
    int32_t pin = -1;
    uint8_t* pinflag = nullptr;         // set when more than one index is pinned
    int32_t precision = BID_FP64;
    int32_t* pidx = nullptr;
    int32_t* bidx = nullptr;
    int32_t* inc = nullptr;
    int32_t* drows = nullptr;
    int32_t* uout = nullptr;
    int32_t* vgl = nullptr;
    HSnode* sn = nullptr;
    HLr* lr = nullptr;
    FGroup* fg = nullptr;
    GCl* gcl = nullptr;
    HTask* uft = nullptr;
    HTask* ubt = nullptr;
    MidCl* mid = nullptr;
    std::vector<int32_t> mid_ptr, ulr_mid;
    std::vector<MidLayout> mid_lay;     // per level (mid clusters' shared memory)
    WideCl* wide = nullptr;
    WideSlice* wslice = nullptr;
    WidePiece* wpiece = nullptr;
    WideAdj* wadj = nullptr;
    std::vector<int32_t> wide_ptr, wide_c;   // wide_c[L] > 0: level L runs the wide kernels
    std::vector<MidLayout> wide_lay;    // per level: staging after the largest slice's pieces
    void* data = nullptr;               // double / float / __nv_bfloat16
    int64_t data_elems = 0;
    double* inb = nullptr;              // update slots (nslots, zero where no child writes)
    std::vector<int32_t> fg_ptr, fg_bytes, fg_nc, fg_wf, fg_wb, ulr_ptr, uf_ptr, ub_ptr, vg_ptr, u_ni_max,
        u_nd_max;
    std::vector<int32_t> fg_nbt;        // level -> most boundary rows of a flat group
    int32_t* sched = nullptr;           // device copy of uf_ptr | ub_ptr | ulr_ptr | vg_ptr (H + 1 each)
    int32_t lev_upper = 0;              // first upper level (only large clusters from there up)
    size_t upper_smem = 0;              // dynamic shared memory of the upper forward kernel
    int64_t ubuf_entries = 0, tbuf_entries = 0, pbuf_entries = 0, nslots = 0, vbuf_entries = 0;
    int32_t ntickets = 0;
    int64_t bytes_pass = 0;             // stored factor bytes read by fwd + bwd
    int64_t alg_bytes_pass = 0;         // nonzero entries only (no padding)
    int32_t vec = 2;
    // dataflow schedule of the flat levels [tree_lev0, tree_lev1) (TreeHost; equal: none)
    int32_t tree_lev0 = 0, tree_lev1 = 0, tree_first = 0, tree_ntask = 0;
    int32_t* tree_idx = nullptr;        // need_f | ptr_f | succ_f | need_b | ptr_b | succ_b
    int64_t tree_off[6] = {0, 0, 0, 0, 0, 0};
    unsigned int* tree_state = nullptr; // counters f (ntask) | b (ntask) | queue f (2) | queue b (2)
    int32_t tree_sc_off = 0, tree_w_off = 0, tree_smem_f = 0, tree_smem_b = 0;
    int32_t tree_cta_f = 0, tree_cta_b = 0;   // resident CTAs per SM
    // masked solve (upload_liveness): live flags per flat group / upper forward
    // task / mid cluster, and the forward results of the all-ones input (y1: ybuf, y1slot:
    // update slots), filled by hsolve_ones
    uint8_t* fg_live = nullptr;
    uint8_t* uf_live = nullptr;
    uint8_t* mid_live = nullptr;
    uint8_t* wide_live = nullptr;
    uint8_t* cl_live = nullptr;         // per cluster
    void* gram = nullptr;               // top-block Gram matrix (storage precision, row stride gram_ld), or NULL
    int32_t gram_s = -1, gram_lev = -1, gram_ld = 0, gram_ni = 0, gram_rows = 1;
    int32_t* top_pos = nullptr;         // HFactorHost::top_pos / top_sptr / top_slot
    int32_t* top_sptr = nullptr;
    int32_t* top_slot = nullptr;
    bool gram_masked = false;           // the masked solve may use it too (the root is live)
    int32_t* fg_mlist = nullptr;        // flat groups of the masked forward launches, level by level
    std::vector<int32_t> fg_mptr;       // level -> range of fg_mlist
    double* y1 = nullptr;
    double* y1slot = nullptr;
    bool ones_ready = false;
    // persistent double-buffered flat launches (k_flat_fwd_pb / k_flat_bwd_pb):
    // per level the grid (0: one CTA per group instead) and the buffer size
    std::vector<int32_t> fgp_grid_f, fgp_grid_b, fgp_buf_f, fgp_buf_b;
};
// Dataflow schedule of the flat groups of the levels [lev0, lev1): the groups
// first .. first + ntask - 1 (tasks, numbered from 0 in group order = lower
// level first) that the persistent solve kernels run in two launches instead
// of one launch per level.  Dependencies on groups outside the range are met
// by the launches before (forward: lower levels) or after (backward) them.
//  forward:  group h waits for need_f[h] signals, one from every group g
//            holding a child of one of its clusters (g writes h's update
//            slots); g signals succ_f[ptr_f[g] .. ptr_f[g+1]);
//  backward: group g waits for need_b[g] signals, one from every group h
//            holding the pivot of a boundary row of one of its clusters (h
//            writes that entry of x); h signals succ_b[ptr_b[h] .. ptr_b[h+1]).
// Forward edges go from a lower to a higher group index, backward edges from a
// higher to a lower one, so handing the groups out in increasing (forward) or
// decreasing (backward) order never makes a group wait for a later one.
// The levels are the longest run from level `from` with no large cluster
// whose largest group fits smem_cap bytes of shared memory; fewer than two
// levels: no schedule (lev1 = lev0 = 0).
struct TreeHost {
    int32_t lev0 = 0, lev1 = 0, first = 0, ntask = 0;
    std::vector<int32_t> need_f, ptr_f, succ_f, need_b, ptr_b, succ_b;
    int32_t sc_off = 0;                 // shared memory: group block | descriptors (sc_off)
    int32_t w_off = 0;                  //   | staged inputs (w_off)
    int32_t smem_f = 0, smem_b = 0;     // bytes of a forward / backward CTA
};
int build_tree_sched(const HFactorHost& F, int acc_bytes, int smem_cap, int from, TreeHost* T);

// Clusters whose subtree holds a pivot with a live vector index
// (vlive[index] != 0; indices beyond vlive are dead): their own pivots, then
// upwards through the update slots (a child's boundary rows write its
// parent's slots).  In a solve whose input is zero on every other index, up
// to a shift c constant on each tree, every other cluster sees the constant
// input -c alone, so its forward results are -c times those of the all-ones
// input (masked solve).
void cluster_liveness(const HFactorHost& F, const std::vector<uint8_t>& vlive, std::vector<uint8_t>* live);
// Clusters whose update slots the masked solve reads: the live ones and the
// dead ones with a live parent (the owner of one of their boundary slots).  A
// dead cluster whose parent is dead writes nothing in the masked forward
// pass: its parent takes the scaled all-ones results without reading slots,
// and the backward pass forms its y as c times the all-ones y.
void cluster_frontier(const HFactorHost& F, const std::vector<uint8_t>& live, std::vector<uint8_t>* send);

int upload_hfactor(const HFactorHost& h, int precision, HFactorDev* d);
// Flags of the masked solve (cluster_liveness with vlive) for the clusters,
// the flat groups and the upper forward tasks, the flat groups each level's
// masked forward launch covers (those holding a cluster of cluster_frontier),
// and room for the all-ones forward results.
int upload_liveness(const HFactorHost& h, const std::vector<uint8_t>& vlive, HFactorDev* d);
void free_hfactor(HFactorDev* d);

// Scratch of one triangular solve (sized by the factor; reused by every solve).
struct HScratch {
    double* xp = nullptr;      // permuted, shifted input (n)
    double* ybuf = nullptr;    // forward result (n)
    double* inb = nullptr;     // update slots (nslots, zeroed); NULL: the factor's own
    double* tbuf = nullptr;    // low-rank products
    double* pbuf = nullptr;    // partial sums of split row chunks
    double* vbuf = nullptr;    // staged backward inputs of the large clusters of a level
    unsigned int* tickets = nullptr;    // zero between solves
    unsigned int* err = nullptr;        // set (nonzero) when a bounded device wait expired
    unsigned int* gbar = nullptr;       // grid barrier of the persistent upper-level kernels
                                        // (2 words, zero initially)
};

// ---------------------------------------------------------------- geometric multigrid
// Alternative elliptic solver for P_1 and P_K (the paper admits any
// preconditioner of S_1 and K there): one V-cycle of geometric multigrid on a
// mesh whose nodes form a regular lattice and whose simplices are the Kuhn
// (Freudenthal) simplices of its cells (2D: every square cut along its "/"
// diagonal; 3D: six tetrahedra around the main diagonal).  Coarse level =
// the lattice points with all indices even; prolongation = P1 interpolation
// (a fine point with odd indices is the midpoint of the coarse points
// floor(i/2) and floor(i/2) + (i mod 2), an edge of the coarse Kuhn
// triangulation), entries whose coarse point is missing from the node set are
// dropped (the heart sub-lattice of P_K); coarse operators A_c = P^T A P
// (Galerkin, symmetrised); smoother: Chebyshev polynomial of degree MG_DEGREE
// in D^-1 A on [MG_LOW lmax, MG_HIGH lmax], lmax from MG_POWER power
// iterations; coarsest level (at most MG_COARSEST points): explicit dense
// inverse, or for the singular S_1 the pseudo-inverse (I - J) E A_pin^-1 E (I - J)
// (last point pinned, E zeroes it, J the mean).
constexpr int MG_DEGREE = 2;
constexpr double MG_LOW = 0.3, MG_HIGH = 1.1;
constexpr int MG_POWER = 20;
constexpr int MG_COARSEST = 512;
constexpr int MG_MAX_LEVELS = 24;

struct MgLevelHost {
    int64_t n = 0;
    CsrHost A;                   // level operator (symmetric)
    std::vector<double> dinv;    // 1 / diag(A)
    CsrHost P, R;                // prolongation (n x n_coarse) and its transpose (absent on the coarsest)
    double lmax = 0.0;           // power-iteration estimate of the largest eigenvalue of D^-1 A
};
struct MgHost {
    std::vector<MgLevelHost> lev;
    std::vector<double> G;       // coarsest-level inverse (nc x nc, row-major)
    int64_t nc = 0;
    bool singular = false;
};
// Lattice of the mesh nodes (coordinates of all N nodes, library order).
struct Lattice {
    int dim = 0;
    double x0[3] = {0, 0, 0}, h[3] = {1, 1, 1};
};
int lattice_of(const double* coords, int64_t n, int dim, Lattice* L);
// Hierarchy for A (rows = the first A.n nodes of the mesh, coords in library
// order); singular: A is the Neumann S_1 (kernel = constants).  EINVAL when
// the nodes are not lattice points or A couples points that are not Kuhn
// neighbours.
int build_mg(const CsrHost& A, const double* coords, const Lattice& L, bool singular, MgHost* out);
// One V-cycle on the host in FP64, the device algorithm's order of operations
// per entry (reference for tests): x = V(b - shift) with shift = mean(b) when
// `project`, x projected onto 1^perp for the singular hierarchy.
void mg_vcycle_host(const MgHost& M, const double* b, bool project, double* x);
// Chebyshev coefficients of level lmax: theta, and (c1, c2) of step 2.
void mg_cheb_coeffs(double lmax, double* theta, double* c1, double* c2);

// A level matrix in sliced ELLPACK (32-row slices) with values in the
// hierarchy's storage type (double or float).
struct MgMat {
    int32_t n = 0, nslices = 0;
    int32_t* sptr = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;
};
// Device hierarchy; matrices, 1/diag, the coarsest inverse and the work
// vectors are stored (and the products accumulated) in FP64 or FP32
// (`precision`); the cycle's input and output vectors are FP64.
struct MgLevelDev {
    int64_t n = 0;
    MgMat A, P, R;
    void* dinv = nullptr;
    double lmax = 0.0;
    void *x = nullptr, *y = nullptr, *b = nullptr, *r = nullptr, *d = nullptr;   // work vectors
    void* e = nullptr;           // this level's V-cycle result (the coarse correction of the level above)
};
struct MgDev {
    std::vector<MgLevelDev> lev;
    void* G = nullptr;
    int64_t nc = 0;
    bool singular = false;
    int precision = BID_FP64;    // BID_FP64 or BID_FP32
    int64_t alg_bytes = 0;       // algorithmic bytes of one V-cycle
};
struct Launch;
int upload_mg(const MgHost& h, int precision, MgDev* d);
void free_mg(MgDev* d);
// x = V-cycle(in - shift), shift = *shift_sum * inv_n when shift_sum != NULL;
// singular hierarchies return x with zero mean.
int launch_mg(const Launch& L, const MgDev& M, const double* in, const double* shift_sum, double inv_n,
              double* x);

// ---------------------------------------------------------------- device scalars
// Scalars of the PCG recurrences, kept on the device so that no kernel needs a
// host round trip.  Reductions are deterministic (fixed order).
struct DevScalars {
    double pq, sumq, alpha;
    double rr, sumr;
    double rz, rz_new, qz, beta;
    double yy, sum_a, sum_b;
    double shift1, shift2;
    double gen[4];
    double tol2;            // tol^2 of the running solve (device-resident loop)
    int iter, max_iter;     // iterations done / allowed
    int go, pad0;           // loop condition when the loop runs from the host
    unsigned int herr, pad1;    // error word of the factor solves (HScratch::err)
    unsigned int ticket[16];
};

// ---------------------------------------------------------------- kernels (device entry)
struct Launch {
    int sms = 152;
    cudaStream_t st = nullptr;
};

// Lambda product / residual (fused): mode 0: q = Lambda p, sums <p,q>, sum(q_U)
// and sets alpha = rz / <p,q>; mode 1: r = Y - Lambda x, sums ||Y||^2, sum(r_U).
int launch_lambda(const Launch& L, int mode, int64_t N, int64_t NH, const SellDev& S1,
                  const SellDev& Si, const double* mH, double gamma, const double* x,
                  double* out, const double* Y, DevScalars* sc, double* partials);
int launch_project(const Launch& L, int64_t N, int64_t NH, double* r, DevScalars* sc,
                   double* partials);
int launch_update(const Launch& L, int64_t N, int64_t NH, double* x, double* r,
                  const double* p, const double* q, DevScalars* sc, double* partials);
int launch_dot_rz(const Launch& L, int64_t n, int64_t N, const double* r, const double* z,
                  const double* q, int flexible, int first, DevScalars* sc,
                  double* partials);
int launch_pupdate(const Launch& L, int64_t n, double* p, const double* z, int first,
                   const DevScalars* sc);
int launch_si_residual(const Launch& L, int64_t NH, const SellDev& Si, const double* rV,
                       const double* z1, double* t);
int launch_si_apply_sum(const Launch& L, int64_t N, int64_t NH, const SellDev& Si,
                        const double* z2, double* w, DevScalars* sc, double* partials);
int launch_sum(const Launch& L, int64_t n, const double* x, double* dst_sum,
               unsigned int* ticket, double* partials);
int launch_axpy_sub(const Launch& L, int64_t n, double* a, const double* b);
int launch_rhs_gate(const Launch& L, int64_t N, int64_t NH, const double* V, double* h,
                    const double* Ist, int stim_on, const double* mH, const bid_params& p,
                    double dt, double* Y);
// Crank-Nicolson Step 1 + Step 3 (S_i (Pi U + V) fused in): Y = [0; m_H (2 gamma V -
// 2 chi (I_ion - I_st)) - S_i (Pi U + V)], h += dt g(V, h); gamma = chi Cm / dt.
int launch_rhs_gate_cn(const Launch& L, int64_t N, int64_t NH, const SellDev& Si, const double* U,
                       const double* V, double* h, const double* Ist, int stim_on, const double* mH,
                       const bid_params& p, double dt, double* Y);
// Strang reaction half step by Heun's method (mode 0: before the diffusion
// step, V -> V* (also to vstar) and Y = [0; g2 m_H V*]; mode 1: after it, from
// 2 Z_V - V* with Z_V in V).
int launch_react_heun(const Launch& L, int mode, int64_t N, int64_t NH, double* V, double* h,
                      double* vstar, const double* Ist, int on0, int on1, double tau, double g2,
                      const double* mH, const bid_params& p, double dt, double* Y);
int launch_normalise(const Launch& L, int64_t N, double* U, const double* m,
                     double msum, DevScalars* sc, double* partials);
// One-thread convergence check of the device-resident PCG loop: first != 0
// resets the iteration count, otherwise it is incremented; the loop continues
// iff ||r||^2 > tol^2 ||Y||^2, the residual is finite, fewer than max_iter
// iterations are done and no factor solve reported an expired wait.  The answer goes to the WHILE condition `h` when
// use_graph != 0, else to sc->go (host-driven loop).
int launch_check(const Launch& L, DevScalars* sc, unsigned long long h, int use_graph, int first);
// The PCG loops run as CUDA graphs with a device-side WHILE condition unless
// the environment sets BID_PCG_GRAPH=0: then the host launches the same
// kernels in the same order and reads the condition after every iteration
// (for profilers that do not see kernels inside graphs with conditional nodes).
bool pcg_graph_enabled();
// x = P^-1 b over a hierarchical factor: forward pass level by level (leaves
// first), then backward pass.  The input entries are b[i] - shift_sum*inv_n
// (shift_sum may be NULL), with the pinned entry set to zero.
int launch_hsolve(const Launch& L, const HFactorDev& F, const double* in,
                  const double* shift_sum, double inv_n, const HScratch& S, double* out);
// Same with one shift per segment (block-diagonal systems): input entry of
// vector index i is b[i] - seg_sum[seg[i]] * seg_inv_n[seg[i]].
// x = P^-1 (b - shift) for an input b that is zero outside the live clusters
// (upload_liveness): the other clusters' forward results are scaled copies of
// the all-ones results (needs hsolve_ones first).  Same result as
// launch_hsolve up to rounding.
int launch_hsolve_masked(const Launch& L, const HFactorDev& F, const double* in, const double* shift_sum,
                         double inv_n, const HScratch& S, double* out);
// the all-ones forward results of a factor with liveness flags (blocking);
// vn: length of the vectors the factor's indices point into
int hsolve_ones(const Launch& L, HFactorDev* F, const HScratch& S, int64_t vn);
// launch_hsolve_masked with one shift per segment (the batched forests)
int launch_hsolve_seg_masked(const Launch& L, const HFactorDev& F, const double* in, const int16_t* seg,
                             const double* seg_sum, const double* seg_inv_n, const HScratch& S, double* out);
bool hsolve_mask_enabled();   // BID_MASK=0 in the environment: plain solves
bool hsolve_flatp_enabled();  // BID_FLATP=1 in the environment: persistent flat launches
bool hsolve_pdl_enabled();    // BID_PDL=0 in the environment: plain stream order
int launch_hsolve_seg(const Launch& L, const HFactorDev& F, const double* in,
                      const int16_t* seg, const double* seg_sum, const double* seg_inv_n,
                      const HScratch& S, double* out);
int hsolve_prepare();   // raise the dynamic shared-memory limit of the kernels
bool hsolve_upper_enabled();   // persistent upper-level kernels in use (after hsolve_prepare)

// ---------------------------------------------------------------- batched form
// Slice s of a batch owns the combined-vector segment [off[s], off[s+1]) laid
// out as a single system ([U_s | V_s]); its heart-indexed arrays (gates,
// stimulus) sit at [hoff[s], hoff[s+1]).
struct BatchHost {
    int S = 0;
    std::vector<int64_t> off, hoff, N, NH;
};
// Factor of a batch: which = 1: the S_1 of every slice (last U unknown of each
// pinned), which = 2: K_m = gamma M_H + S_m of every slice; one cluster tree
// per slice (leaf size leaf[s]), vector indices in the combined layout.
int build_batch_factor(const std::vector<const AssembledHost*>& A, const BatchHost& lay, int which,
                       double gamma, const HBuildOpts& base, const std::vector<int32_t>& leaf,
                       HFactorHost* F);

struct BCta {              // CTA task: slice s, range [a, b) (elements or tiles)
    int32_t s, a, b, pad;
};
struct BTasks {
    const BCta* t;
    const int32_t* ptr;    // slice s owns tasks [ptr[s], ptr[s+1])
    int n;
};
struct BGeom {
    int S;
    const int32_t *off, *N, *NH, *hoff;
    const double *invN, *msum;
    const double* mdiag;   // lumped m at U positions, m_H at V positions
};
// 32-row SELL tiles of every slice's S_1 (sp1/col1/val1) and S_i (sp2/...;
// empty beyond the heart rows); tile t of slice s covers local rows
// 32 (t - tile0[s]) ...; columns are local to the slice.
struct BSell {
    const int32_t *sp1, *sp2, *tile0, *col1, *col2;
    const double *val1, *val2;
};
// Per-slice PCG scalars (device arrays of S entries).
struct BScal {
    double *pq, *sumq, *alpha, *rr, *sumr, *rz, *beta, *yy, *sumb, *gen, *suma;
    double* tol2;          // one value
    int32_t *iter, *active, *mask, *maxit;
    int32_t* go;           // loop condition when the loop runs from the host
    unsigned int* ticket;  // one per kernel kind
};
struct MsParamsB {
    double v_rest, span, tau_in, tau_out, tau_open, tau_close, v_gate, Cm, chi, gamma, dt;
};
int blaunch_lambda(const Launch& L, int mode, const BGeom& g, const BSell& A, const BTasks& T,
                   double gamma, const double* x, double* out, const double* Y, const BScal& c,
                   double* partials);
int blaunch_project(const Launch& L, const BGeom& g, const BTasks& T, double* r, const BScal& c,
                    double* partials);
int blaunch_update(const Launch& L, const BGeom& g, const BTasks& T, double* x, double* r,
                   const double* p, const double* q, const BScal& c, double* partials);
int blaunch_dot_rz(const Launch& L, const BGeom& g, const BTasks& T, const double* r,
                   const double* z, const double* q, int flexible, const BScal& c,
                   double* partials);
int blaunch_pupdate(const Launch& L, const BTasks& T, double* p, const double* z, const BScal& c);
int blaunch_si_residual(const Launch& L, const BGeom& g, const BSell& A, const BTasks& T,
                        const double* r, const double* z, double* t);
int blaunch_si_apply_sum(const Launch& L, const BGeom& g, const BSell& A, const BTasks& T,
                         const double* z, double* w, const BScal& c, double* partials);
int blaunch_sum_u(const Launch& L, const BGeom& g, const BTasks& T, const double* x, double* dst,
                  const BScal& c, double* partials);
int blaunch_axpy_sub_u(const Launch& L, const BGeom& g, const BTasks& T, double* z,
                       const double* b);
int blaunch_rhs_gate(const Launch& L, const BGeom& g, const BTasks& T, const double* X, double* h,
                     const double* Ist, int stim_on, const bid_params& p, double dt, double* Y);
int blaunch_normalise(const Launch& L, const BGeom& g, const BTasks& T, double* X, const BScal& c,
                      double* partials);
int blaunch_check(const Launch& L, int S, const BScal& c, unsigned long long h, int use_graph,
                  int first);

// ---------------------------------------------------------------- learned guess
int guess_ready(const bid_guess* G);
int guess_push(bid_guess* G, const double* U, const double* V, cudaStream_t st);
// *X0 points at the guess's own buffer (N + N_H)
int guess_predict(bid_guess* G, const double* U, const double* V, double** X0, cudaStream_t st);
int guess_policy(const bid_guess* G);
int guess_choose(bid_guess* G);                    // arm of the next step (policy 1)
void guess_record(bid_guess* G, int arm, int iters);

// ---------------------------------------------------------------- handles
}  // namespace bid

struct bid_system {
    bid::AssembledHost host;
    bid_params params{};
    bid::SellDev S1, Si;
    double* m = nullptr;      // device lumped mass (N)
    double* mH = nullptr;     // device lumped heart mass (N_H)
    double msum = 0.0;
    int sms = 152;
};

struct bid_precond {
    bid_system* sys = nullptr;
    bid_precond_opts opts{};
    double gamma = 0.0;
    bid::HFactorDev F1, FK;
    // work vectors (device)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double *z1b = nullptr, *t = nullptr, *w = nullptr, *ytmp = nullptr, *xs = nullptr;
    double* vstar = nullptr;                  // Strang scheme: V after the first reaction half step
    bool mg = false;                          // P_1, P_K by multigrid V-cycles (M1, MK), not F1, FK
    bid::MgDev M1, MK;
    bid::HScratch hs;
    double* partials = nullptr;
    bid::DevScalars* sc = nullptr;
    bid::DevScalars* host_pinned = nullptr;   // pinned host mirror of the scalars
    bid_precond_stats stats{};
    // device-resident PCG loop: one graph per preconditioner (built on first use)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;               // private stream used for capture only
    int g_prologue = 0, g_body = 0;           // kernels per prologue / per iteration
};

struct bid_batch {
    int S = 0;
    std::vector<bid_system*> sys;
    bid::BatchHost lay;
    bid_precond_opts opts{};
    std::vector<int32_t> leaf;
    double gamma = 0.0;
    int sms = 152;
    bid::HFactorDev F1, FK;
    bid::HScratch hs;
    // device geometry, tiles and tasks
    int32_t *d_off = nullptr, *d_N = nullptr, *d_NH = nullptr, *d_hoff = nullptr;
    double *d_invN = nullptr, *d_msum = nullptr, *mdiag = nullptr;
    int16_t* seg = nullptr;
    int32_t *sp1 = nullptr, *sp2 = nullptr, *tile0 = nullptr, *col1 = nullptr, *col2 = nullptr;
    double *val1 = nullptr, *val2 = nullptr;
    bid::BCta *vt = nullptr, *lt = nullptr, *ht = nullptr;
    int32_t *vptr = nullptr, *lptr = nullptr, *hptr = nullptr;
    int nvt = 0, nlt = 0, nht = 0;
    // work vectors (combined layout)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *xs = nullptr, *ytmp = nullptr;
    double *z1b = nullptr, *t = nullptr, *w = nullptr, *partials = nullptr;
    double* dscal = nullptr;       // per-slice double scalars
    int32_t* iscal = nullptr;      // per-slice int scalars
    unsigned int* tickets = nullptr;
    void* host_pinned = nullptr;   // mirror of dscal + iscal
    bid::BScal sc{};
    bid_precond_stats stats{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;
    int g_prologue = 0, g_body = 0;
    bid::BGeom geom() const {
        return bid::BGeom{S, d_off, d_N, d_NH, d_hoff, d_invN, d_msum, mdiag};
    }
    bid::BSell sell() const { return bid::BSell{sp1, sp2, tile0, col1, col2, val1, val2}; }
    bid::BTasks vtasks() const { return bid::BTasks{vt, vptr, nvt}; }
    bid::BTasks ltasks() const { return bid::BTasks{lt, lptr, nlt}; }
    bid::BTasks htasks() const { return bid::BTasks{ht, hptr, nht}; }
};
