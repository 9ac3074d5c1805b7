// ipm_internal.h -- plan parameters shared by the host planner and kernels.
#pragma once
#include <stdint.h>
#include <stddef.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/ipm.h"

namespace ipm {

constexpr int RMAX = 6;              // most Fourier primes a plan may use
constexpr int PRIME_ORDER_LOG2 = 21; // every prime p satisfies 2^21 | p - 1
constexpr int KMAX_LOG2 = 11;        // K <= 2048 digits per coefficient
constexpr int MMAX = 62;             // digit width, |digit| <= 2^(M-1) < 2^63

// Dynamic shared memory: hard limit per block (sm_103a allows 227 KB), and
// the sizes below which 3 forward / 2 inverse CTAs fit on one SM.
constexpr size_t SMEM_BLOCK_MAX = 227 * 1024;
constexpr size_t SMEM_FWD_MAX = SMEM_BLOCK_MAX;
constexpr size_t SMEM_INV_MAX = SMEM_BLOCK_MAX;
constexpr size_t SMEM_MID_MAX = SMEM_BLOCK_MAX;
constexpr size_t SMEM_FWD_3PERSM = 74 * 1024;
constexpr size_t SMEM_INV_2PERSM = 112 * 1024;

constexpr int THREADS_FWD = 256;
constexpr int THREADS_MID = 512;
constexpr int THREADS_INV = 512;
constexpr int THREADS_OUTER = 256;
constexpr int OUTER_TILE_WORDS = 8192;  // outer-pass tile: Y1b rows x W words

// Tensor-core radix-16 stage tables (IPM_TENSOR_STAGES): per prime, the A
// fragments of the forward and of the inverse radix-16 DFT matrix in byte
// slices (ntt_stages.cuh, stage_tc16), 1024 words each.
constexpr int TC_FRAG_WORDS = 2048;

// Middle-pass tile rows (passes.cuh, mid_tile): for slices of S < 32
// columns, one empty row after every 2^pl rows, 2^pl the radix of the last
// stage of the length-2^logY1a column transform (the register stages split
// log2 L into ceil(log2 L / 4) stages as evenly as possible, the last one
// smallest); 0 for S >= 32, whose rows need no padding: a warp's accesses
// then cover whole rows.
__host__ __device__ inline int mid_pad_log(int logY1a, int S) {
    if (S >= 32 || logY1a < 1) return 0;
    const int nst = (logY1a + 3) / 4;
    return logY1a / nst;
}

// Row pitch (words) of a middle tile: S (padded rows, or S >= 32), else the
// odd S + 1 (a one-row column, no padding).
__host__ __device__ inline int mid_pitch(int S, int pl) { return pl || S >= 32 ? S : S + 1; }

// Offsets (uint2 entries) of the per-stage twiddle blocks of a compact
// table for a length-2^logL transform: stage i at off[i], 2 (Lc_i + R_i)
// entries; returns the total.
__host__ __device__ inline int stage_blocks(int logL, int (&off)[8]) {
    const int nst = (logL + 3) / 4;
    const int base = nst ? logL / nst : 0, extra = nst ? logL % nst : 0;
    int at = 0, logLc = logL;
    for (int i = 0; i < nst; ++i) {
        const int b = base + (i < extra ? 1 : 0);
        off[i] = at;
        at += 2 * ((1 << logLc) + (1 << b));
        logLc -= b;
    }
    return at;
}

// Device error word bits.
constexpr int ERRBIT_BOUND = 1;      // an input coefficient >= 2^bits
constexpr int ERRBIT_INTERNAL = 2;   // recombination top limb not a sign word
constexpr int ERRBIT_MISMATCH = 4;   // IPM_VALIDATE: c(t) != a(t) b(t) mod 2^61 - 1
constexpr int ERRBIT_TIMEOUT = 8;    // IPM_PERSISTENT: a dependency wait ran out

// Randomised product check (ipm_validate.cu): blocks and threads of the
// evaluation kernels; the scratch holds 3 x VAL_BLOCKS partial sums.
constexpr int VAL_BLOCKS = 1216;  // 8 per SM: 64 warps in flight
constexpr int VAL_THREADS = 256;

// Per-prime constants.  Twiddle tables hold (w, floor(w * 2^32 / p)) pairs
// for Shoup's precomputed-quotient multiplication.
struct PrimeConst {
    uint32_t p;        // prime, 2^29 < p < 2^30, p = 1 mod 2^21
    uint32_t p2;       // 2p
    uint32_t mont;     // -p^{-1} mod 2^32 (Montgomery REDC)
    uint32_t one_s;    // floor(2^32 / p): Shoup quotient of w = 1
    uint32_t c32;      // 2^32 mod p
    uint32_t c32_s;    // its Shoup quotient
    uint32_t scale;    // 2^32 * (2 Y K)^{-1} mod p (inverse-transform scale)
    uint32_t scale_s;
    const uint2 *ty_f; // omega_Y^e,     e < Y   (forward y twiddles)
    const uint2 *ty_i; // omega_Y^{-e},  e < Y   (inverse y twiddles)
    const uint2 *t1_f; // omega_Y1^e,    e < Y1  (compact table of the middle pass)
    const uint2 *t1_i; // omega_Y1^{-e}, e < Y1
    const uint2 *tx_f; // theta^e,       e < 2K  (theta: primitive 2K-th root)
    const uint2 *tx_i; // theta^{-e},    e < 2K
    const uint2 *untw; // scale * theta^{-j}, j < K
};

// Everything one product needs on the device (passed by value, < 4 KB).
struct KParams {
    int64_t na, nb, nc;   // coefficient counts of a, b, c
    int32_t la, lb, lc;   // limb strides
    uint32_t bits_a, bits_b;
    int32_t K, logK, M, N, r;
    int64_t Y, Y1, Y2;
    int32_t logY, logY1, logY2, S, logS;
    int32_t mid_tables_in_smem;  // middle pass keeps its omega_Y1 tables in shared memory
    // Three-level split of the middle transform (Y1 = Y1a * Y1b, Y1b > 1):
    // an outer pass does the length-Y1b transforms over i1b (rows i1a +
    // Y1a i1b) and the twiddle omega_Y1^{i1a k1b}; the middle pass then
    // works on length-Y1a columns.  Y1b = 1: no split.
    int64_t Y1a, Y1b;
    int32_t logY1a, logY1b, S2, logS2;  // S2: outer-pass tile width in words
    PrimeConst pc[RMAX];
    // Garner: ginv[t][s] = p_s^{-1} mod p_t (s < t), with Shoup quotients.
    uint32_t ginv[RMAX][RMAX];
    uint32_t ginv_s[RMAX][RMAX];
    // m = prod p_t as r little-endian 32-bit words (fits: each p < 2^30).
    uint32_t m_words[RMAX];
    uint32_t *Z;          // workspace: r x 2 x Y x 2K words
    int *err;             // device error word
    int32_t batch_index;  // batched launches: index of this product's operands
    // IPM_TENSOR_STAGES: r x TC_FRAG_WORDS fragment words (prime t at
    // t * TC_FRAG_WORDS), or null for the integer stages
    const uint32_t *tcfrag;
};

// Host-side plan record for one shape.
// Kronecker balancing: the product a*b is computed as the product of the
// packed polynomials A'(z) = sum_k A'_k z^k, A'_k = sum_{u<s} a_{ks+u} 2^{uw}
// (likewise B'), whose coefficient C'_k = sum_{t<2s-1} D_{k,t} 2^{tw} holds
// the partial sums D_{k,t} = sum_{i+j=k, u+v=t} a_{is+u} b_{js+v} in
// balanced w-bit slots; c_{ks+t} = D_{k,t} + D_{k-1,t+s}.  The packed
// operands and product live after the transform workspace.
constexpr int KRON_MAX = 16;
constexpr int KRON_WMAX = 128;
struct KronPlan {
    int32_t s;                 // coefficients per packed coefficient (1 = none)
    int32_t w;                 // slot width in bits
    int64_t na, nb, nc;        // the original shape
    int32_t la, lb, lc;
    uint32_t bits_a, bits_b;
    size_t off_a, off_an, off_b, off_bn, off_c, off_cn;  // word offsets from Z
};

// Kronecker substitution (ipm_ks.cu): the product read off the integer
// product a(2^s) b(2^s), s = 32 w, w = lc + 3 limbs per slot; the integer
// product is the transform product (kp) of the operands' digit
// polynomials (na w and nb w coefficients of 32 bits).  Buffers after the
// transform workspace (word offsets from Z): the digit polynomials, their
// product (lc' limbs per digit), and per slot t <= nc the low s bits L_t,
// the high part H_t (int64) and the top bit of L_t.
struct KsPlan {
    int32_t on;
    int32_t w;
    int64_t na, nb, nc;
    int32_t la, lb, lc;
    uint32_t bits_a, bits_b;
    size_t off_a, off_an, off_b, off_bn, off_c, off_cn, off_L, off_H, off_g;
};

// The Karatsuba family (ipm_kara.cu): `levels` levels over y, operands
// padded to n2 = m 2^levels, 3^levels schoolbook leaves of m x m
// coefficients (kp describes one leaf product: m, m, lla / llb limbs,
// bits + levels, output stride lci).  Buffers after nothing else (word
// offsets from Z): leaf operands and signs, then the products of every
// level d = 1 .. levels (3^d products of 2 n2 / 2^d - 1 coefficients, lci
// limbs each) and their signs; level 0 is the output c.
constexpr int KARA_MAX_LEVELS = 4;
struct KaraPlan {
    int32_t levels;  // 0: not this family
    int64_t n2, m;
    int64_t na, nb, nc;
    int32_t la, lb, lc, lla, llb, lci;
    uint32_t bits_a, bits_b;
    size_t off_a, off_an, off_b, off_bn;
    size_t off_lev[KARA_MAX_LEVELS + 1], off_levn[KARA_MAX_LEVELS + 1];
};

// The big-prime form (ipm_bigp.cu): one generalized Fermat prime
// p = (2^63 + 2^53)^2 + 1 instead of r word primes and CRT.  Elements are
// 128-bit words; the workspace (from Z, 16-byte units) holds both operands'
// Y x 2K arrays; the tables (device, built by the plan) hold theta^j,
// scale theta^-j, omega_K^(+-e) and omega_Y^(+-e) at the tab_* offsets.
struct BigpPlan {
    int32_t on;
    int32_t K, logK, M, N;
    int64_t Y;
    int32_t logY;
    int64_t na, nb, nc;
    int32_t la, lb, lc;
    uint32_t bits_a, bits_b;
    size_t off_xa, off_xb;  // in 128-bit units from Z
    size_t tab_theta, tab_untw, tab_wk, tab_wk_i, tab_wy, tab_wy_i, table_entries;
    uint64_t scale_lo, scale_hi, half_lo, half_hi;
    const void *dtab;
};
// Tables (host, 64-bit words) and the 4H < p test of the big-prime form.
void bigp_tables(BigpPlan &b, std::vector<uint64_t> &words);
bool bigp_bound_ok(int64_t mn, int K, int M);

struct ShapePlan {
    ipm_plan_info info;
    BigpPlan bp;          // on = 0: not the big-prime form
    KaraPlan ka;          // levels = 0: not the Karatsuba family
    KsPlan ks;            // on = 0: not the Kronecker-substitution family
    KronPlan kr;          // s = 1: no packing (kp describes the product itself)
    bool school;          // schoolbook family: only kp's shape fields and err are used
    KParams kp;           // pointers filled in by ipm_plan
    size_t smem_fwd, smem_mid, smem_inv, smem_outer;
    size_t z_words;       // workspace words
    size_t table_words;   // table uint2 entries per prime
};

// Planner (host only).  Fills sp (minus device pointers) or returns an error.
ipm_status choose_plan(const ipm_shape &shape, const ipm_params *params, ShapePlan &sp);
// Slot width of Kronecker packing for a shape (KronPlan).
int kron_slot_width(const ipm_shape &shape);
// Counts launches of this library's kernels (ipm_launch_count).
void note_launches(int n);

// Learned dispatch for n shapes (ipm_mlp.cu): params per shape and their
// source (0 planner: params all zero, 1 tuning table, 2 model).
ipm_status dispatch_params(const ipm_shape *shapes, int32_t n, ipm_params *out, int32_t *src);

// Builds the per-prime tables for sp into host memory `tab` (r blocks of
// sp.table_words uint2 entries) and fills the scalar constants of sp.kp.
void build_tables(ShapePlan &sp, uint2 *tab);

// The tensor-core stage tables of primes[0..r) into out (r x TC_FRAG_WORDS
// words).
void build_tc_fragments(const uint32_t *primes, int r, uint32_t *out);

// Table block offsets (uint2 entries) within one prime's block.
struct TableLayout {
    size_t ty_f, ty_i, t1_f, t1_i, tx_f, tx_i, untw, total;
};
TableLayout table_layout(int64_t Y, int64_t Y1, int32_t K);

// Kernel launchers (ipm_kernels.cu).
int launch_forward(const KParams &kp, size_t smem, const uint32_t *a, const uint8_t *an,
                   const uint32_t *b, const uint8_t *bn, void *stream);
int launch_middle(const KParams &kp, size_t smem, void *stream);
// SMs of the current device (cached per device), and the middle-pass tiles
// of one product (column slices x Y2 x Y1b x primes).
int sm_count();
int middle_tiles(const KParams &kp);
int launch_inverse(const KParams &kp, size_t smem, uint32_t *c, uint8_t *cn, void *stream);
int launch_outer(const KParams &kp, size_t smem, bool forward, void *stream);
// The launch sequence of the transform product kp describes (forward,
// [outer], middle, [outer inverse], inverse).  Returns 0 or -1.
int launch_transform_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                             const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
// Pack, transform product of the packed operands, unpack (ipm_kron.cu).
int launch_kron_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
// Leaf operands, batched schoolbook leaves, level-by-level combination
// (ipm_kara.cu); `count` equal-shape schoolbook products back to back
// (ipm_school.cu).
int launch_kara_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
int launch_school_batch(const KParams &kp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, int64_t count, void *stream);
// The big-prime product (ipm_bigp.cu).
int launch_bigp_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
// Pack, integer product of the digit polynomials, unpack (ipm_ks.cu).
int launch_ks_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                      const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
// One whole product: launch_kron_product when sp.kr.s > 1, launch_ks_product
// for the Kronecker-substitution family, else launch_transform_product.
int launch_product(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                   const uint8_t *bn, uint32_t *c, uint8_t *cn, void *stream);
// The schoolbook family (ipm_school.cu): limits, shared memory, launch.
constexpr int SCHOOL_MAX_COLUMNS = 256;                   // La + Lb
constexpr double SCHOOL_MAX_LIMB_PRODUCTS = 134217728.0;  // na nb La Lb <= 2^27
size_t school_smem(const KParams &kp);
int launch_school(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b, const uint8_t *bn,
                  uint32_t *c, uint8_t *cn, void *stream);
// Products a batched call runs one at a time (split, packed or schoolbook).
inline bool runs_alone(const ShapePlan &sp) {
    return sp.school || sp.kp.Y1b > 1 || sp.kr.s > 1 || sp.ks.on || sp.ka.levels || sp.bp.on;
}
int set_kernel_attributes();
// Evaluation point for a seed, and the check c(t) = a(t) b(t) mod 2^61 - 1
// of one product laid out as I describes (ERRBIT_MISMATCH into *err).
uint64_t validation_point(uint64_t seed);
int launch_validate(const ipm_plan_info &I, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                    const uint8_t *bn, const uint32_t *c, const uint8_t *cn, uint64_t t, uint64_t *part, int *err,
                    void *stream);
// The same check for every product of a batched call, in two launches: one
// warp per item (a chunk of up to VAL_ROWS rows of one operand of one
// product, weighted by t^row0), then one thread per product.  Built once
// by ipm_plan for the plan's fixed point t.
constexpr int VAL_ROWS = 128;
struct ValItem {
    int32_t product, operand;  // operand 0: a, 1: b, 2: c
    int64_t row0;
    int32_t rows, limbs;
    uint64_t t_row0;           // t^row0 mod 2^61 - 1
};
struct ValBatch {
    const ValItem *items = nullptr;  // device
    int64_t nitems = 0;
    const int64_t *first = nullptr;  // device: first[3 i + o] = first item of product i, operand o; first[3 n] = nitems
    int32_t nproducts = 0;
    uint64_t *part = nullptr;        // device: one partial sum per item
    uint64_t t = 0;
};
// Host: t^e mod 2^61 - 1 (the item weights).
uint64_t pow61_host(uint64_t t, uint64_t e);
int launch_validate_batch(const ValBatch &vb, const ipm_operands *ops, int *err, void *stream);
// The same passes with every radix-16 stage on the tensor cores
// (ipm_kernels_tc.cu); the launchers above call these when kp.tcfrag is set.
int set_kernel_attributes_tc();
int launch_forward_tc(const KParams &kp, size_t smem, const uint32_t *a, const uint8_t *an,
                      const uint32_t *b, const uint8_t *bn, void *stream);
int launch_middle_tc(const KParams &kp, size_t smem, void *stream);
int launch_inverse_tc(const KParams &kp, size_t smem, uint32_t *c, uint8_t *cn, void *stream);
int launch_outer_tc(const KParams &kp, size_t smem, bool forward, void *stream);

// One group of a batched call: products that share the kernel variants,
// launched as three ragged grids.  items[p][b] = (index into params, tile).
// A run of a group's forward and inverse items whose products share (K,
// log2 Y2): items [f0, f0 + nf) of the forward list and [i0, i0 + ni) of the
// inverse list (K = 0: products of shapes without a compiled kernel).
struct BatchRun {
    int32_t K, logY2;
    unsigned f0, nf, i0, ni;
};
constexpr int BATCH_RUNS_MAX = 16;
struct BatchLaunch {
    const KParams *params;    // device array
    const uint2 *items[3];    // device arrays, one per pass
    unsigned nitems[3];
    size_t smem[3];           // largest tile of the group, per pass
    bool fwd_small, mid_tables, inv_small;
    int32_t nruns;            // 0: one generic launch per pass
    BatchRun runs[BATCH_RUNS_MAX];
};
int launch_batch(const BatchLaunch &bl, const ipm_operands *ops, void *stream);
// ipm_kernels_batch.cu: batched forward / inverse kernels compiled for fixed
// (K, log2 Y2)
bool batch_shape_compiled(int K, int logY2);
int set_kernel_attributes_batch();
int launch_batch_run(bool fwd, int K, int logY2, const KParams *params, const ipm_operands *ops,
                     const uint2 *items, unsigned n, size_t smem, void *stream);

// IPM_PERSISTENT (ipm_persist.cu): a batched call as one persistent launch
// over a device work queue.  Segment = a run of consecutive items (one
// product's tiles of one phase) starting at queue index `start`.
constexpr size_t PERSIST_WINDOW_WORDS = (size_t)8 << 20;  // 32 MiB of workspace per pipeline window
constexpr size_t PERSIST_SMEM_MAX = SMEM_BLOCK_MAX - 256;  // dynamic shared memory (room for the static part)
constexpr size_t PERSIST_SMEM_SMALL = 112 * 1024;          // two 256-thread blocks per SM below this
constexpr uint64_t PERSIST_WAIT_US_DEFAULT = 2000000;     // 2 s per dependency wait
constexpr int PERSIST_CHUNK = 4;  // tiles per queue entry
struct PersistSeg {
    int64_t start;  // first queue entry (chunk) of the segment
    int32_t product, phase, tiles, pad;
};
struct PersistControl {
    unsigned long long head;  // next queue index
    int abort;                // set when a wait timed out
    int pad;
};
struct PersistLaunch {
    const KParams *params;    // device, one per product of the plan (batch_index = product)
    const PersistSeg *segs;   // device
    int nseg;
    int64_t nitems;
    const int *need;          // device: tiles per (product, phase)
    PersistControl *ctl;      // device: control block, then the per-(product, phase) counters
    int *done;
    size_t ctl_bytes;         // bytes to clear before each launch (control block and counters)
    unsigned blocks;
    size_t smem;
    long long wait_cycles;
};
void persist_schedule(const std::vector<ShapePlan> &shapes, const std::vector<int> &members,
                      std::vector<PersistSeg> &segs, std::vector<int> &need, int64_t &nitems);
int persist_blocks(size_t smem);
int set_kernel_attributes_persist();
int launch_persistent(const PersistLaunch &pl, const ipm_operands *ops, void *stream);
int64_t launches_so_far();

}  // namespace ipm
