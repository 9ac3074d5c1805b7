/*
 * ipm.h -- exact dense integer polynomial multiplication on one GB300 GPU.
 *
 * Method: "Parallel Integer Polynomial Multiplication" (Chen, Covanov,
 * Mansouri, Moreno Maza, Xie, Xie; arXiv 1612.05778), in the form its §4
 * implements (several machine-word Fourier primes and Chinese remaindering,
 * "CVL_p^2"):
 *
 *   1. DetermineBase (§2): N = K*M, beta = 2^M, K a power of two.
 *   2. BivariateRepresentation (§2): every coefficient a_i becomes
 *      sum_{j<K} a_{i,j} beta^j with balanced digits a_{i,j}.
 *   3. CyclicConvolution / NegacyclicConvolution (§2.1): C^-(x,y) = A*B
 *      mod (x^K - 1) and C^+(x,y) = A*B mod (x^K + 1), by two-dimensional
 *      number-theoretic transforms over each prime p_t (the negacyclic one
 *      after the twist x -> theta*x, theta a primitive 2K-th root of unity).
 *   4. Chinese remaindering over the primes (§4) of the per-digit values
 *      c_{i,j} = (c^-_{i,j} + c^+_{i,j})/2 and c_{i,j+K} = (c^-_{i,j} -
 *      c^+_{i,j})/2, which is RecoveringProduct's step 3 (§2.2) written per
 *      digit, then the shift-and-add c_i = sum_j c_{i,j} 2^{Mj} with carry
 *      propagation.
 *
 * Number format (§2.3 stores coefficient i of a in words [i*ceil(N/w),
 * (i+1)*ceil(N/w)); here w = 32 and magnitudes are sign-magnitude):
 *   - coefficient i of a occupies 32-bit little-endian limbs
 *     a[i*La .. (i+1)*La) holding |a_i|, La = ceil(bits_a / 32);
 *   - a_neg[i] is 1 when a_i < 0 and 0 otherwise (-0 is accepted);
 *   - |a_i| < 2^bits_a is required (checked on the device: IPM_ERR_BOUND);
 *   - the product c has (deg_a + deg_b + 1) coefficients with stride
 *     Lc = ceil((bits_a + bits_b + ceil(log2(min(deg_a, deg_b) + 1))) / 32)
 *     limbs (ipm_plan_info.lc); output zero always has c_neg = 0 and every
 *     limb above a coefficient's magnitude is written as 0.
 *
 * Ownership: the caller owns every operand buffer.  A plan owns its
 * device workspace and tables.  Calls on a plan are ordered on the stream
 * given and are asynchronous unless IPM_SYNC is set; one plan must not be
 * used by two calls that overlap in time (they share the workspace).
 *
 * Errors: argument errors are returned at once.  Errors found on the device
 * (an input above its bit bound) are recorded in a per-plan device word and
 * returned by ipm_sync(), or by the call itself when IPM_SYNC is set.
 * Nothing is ever reported by trapping the GPU.
 *
 * Speed: some tile shapes run kernels compiled for that shape, which are
 * 10-30% faster than the general ones with the same results: single
 * products whose plan has (K, Y2, M) = (32, 128, 33), (128, 32, 33) or
 * (128, 32, 17) in the forward and inverse passes and (S, Y1a, K) = (4,
 * 4096, 32), (8, 2048, 128) or (16, 1024, 128) in the middle pass (for
 * example d = 2^18 with 1024-bit and d = 2^15 with 4096-bit coefficients),
 * and, in the forward and inverse passes of batched calls, products with
 * (K, Y2) = (64, 32), (64, 64), (128, 32), (32, 32), (32, 64), (32, 128),
 * (16, 128) or (16, 64).  ipm_get_info shows a plan's K, Y2, S.
 */
#ifndef IPM_H
#define IPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ipm_plan_s *ipm_plan_t;

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef void *ipm_stream_t;

typedef enum {
    IPM_OK = 0,
    IPM_ERR_ARG = 1,          /* invalid argument or shape */
    IPM_ERR_BOUND = 2,        /* an input coefficient is >= 2^bits */
    IPM_ERR_NOMEM = 3,        /* device or host allocation failed */
    IPM_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    IPM_ERR_TIMEOUT = 5,      /* a bounded device wait ran out */
    IPM_ERR_UNSUPPORTED = 6,  /* shape outside what the plan tables support */
    IPM_ERR_MISMATCH = 7      /* a validated product failed its random check */
} ipm_status;

/* Plan flags. */
#define IPM_SYNC 1u           /* calls synchronise and return device errors */
#define IPM_COSTMODEL 2u      /* learned dispatch picks each shape's plan (see
                                 ipm_set_cost_model); ignored with params */
#define IPM_GRAPH 4u          /* batched calls replay one CUDA graph of their
                                 grouped launches (see ipm_mul_batched) */
#define IPM_TENSOR_STAGES 8u  /* every radix-16 transform stage runs as 8-bit
                                 byte-slice matrix products with 32-bit
                                 accumulation on the INT8 tensor cores
                                 (mma.sync .u8), reduced exactly mod p;
                                 bit-identical output.  Applies to products
                                 launched one at a time (ipm_mul, the host-
                                 buffer calls, batched products that run
                                 alone); grouped batch launches keep the
                                 integer stages.  A GPU formulation of the
                                 DFTs of §2.1; the paper has no counterpart. */
#define IPM_PERSISTENT 32u    /* batched calls run as ONE persistent launch over
                                 a device work queue (see ipm_mul_batched) */
#define IPM_VALIDATE 16u      /* every product is checked on the GPU after it
                                 runs (ipm_validate's test: at a fresh random
                                 point for ipm_mul and the host-buffer calls,
                                 at the plan's fixed random point, in two
                                 launches for all products, for batched
                                 calls); a failure is returned as
                                 IPM_ERR_MISMATCH by ipm_sync. */

/* One product shape: a has deg_a+1 coefficients with |a_i| < 2^bits_a. */
typedef struct {
    int64_t deg_a, deg_b;
    uint32_t bits_a, bits_b;  /* 1 .. 65536 */
} ipm_shape;

/*
 * Optional overrides of the planner's choices (0 = let the planner choose).
 * Every valid choice gives the same exact product.
 *   K : number of base-2^M digits per coefficient (power of two, 2..2048)
 *   M : digit width in bits (2..62); needs K*M >= max(bits_a,bits_b)+1
 *   r : number of 30-bit Fourier primes (1..6); needs prod p > 4H (§2.1)
 *   y2: rows per forward/inverse tile (power of two dividing Y)
 *   s : columns per middle-pass tile (power of two dividing 2K)
 *   y1b: split the middle transform in two (power of two > 1 dividing Y/y2)
 *   kron: Kronecker balancing (§3, footnote on balancing): 0 or 1 = none;
 *        2, 4, 8 or 16 = pack this many consecutive coefficients of a and of
 *        b into one coefficient with slots of w = bits_a + bits_b +
 *        ceil(log2 min(na, nb)) + 1 bits (w <= 128), multiply the packed
 *        polynomials with the other parameters, and decode the slots.  For
 *        small coefficients at large degree, where the y transform dominates.
 *   school: 1 = the schoolbook family instead of the transform path:
 *        c_k = sum a_i b_{k-i} by direct 32-bit limb products, one block per
 *        output coefficient (small products only: La + Lb <= 256 and
 *        na nb La Lb <= 2^27); the other fields must then be 0.
 *   ks: 1 = Kronecker substitution (§1, §4: the comparison method KS_s):
 *        c is read off the integer product a(2^s) b(2^s), s = 32 (Lc + 3),
 *        whose digit polynomials (na (Lc+3) and nb (Lc+3) coefficients of
 *        32 bits) are multiplied by the transform path (K, M, r, y2, s and
 *        y1b then apply to that product; kron and school must be 0).  Needs
 *        (na + nb) (Lc + 3) - 1 <= 2^21 (IPM_ERR_UNSUPPORTED otherwise).
 *   kara: L >= 1 = the Karatsuba family: L levels of Karatsuba's
 *        three-product recursion over y (§1 lists Karatsuba among the plain
 *        methods), the schoolbook kernel at the leaves (L <= 4; the leaf
 *        operands, of bits + L bits, must fit the schoolbook limits); the
 *        other fields must then be 0.
 *   bigp: 1 = the big-prime form (§3.1, §4): the same two convolutions
 *        modulo ONE generalized Fermat prime p = (2^63 + 2^53)^2 + 1 instead
 *        of several 30-bit primes and CRT (K may be set; the planner takes
 *        the smallest K with 4H < p and Y <= 2^21; the other fields must be
 *        0).  Simple radix-2 kernels: meant for small products.
 */
typedef struct {
    int32_t K, M, r, y2, s, y1b, kron, school, ks, kara, bigp;
} ipm_params;

/* What a plan chose (ipm_choose / ipm_get_info). */
typedef struct {
    int64_t na, nb, nc;       /* coefficient counts of a, b and c */
    int32_t la, lb, lc;       /* limb strides of a, b and c */
    int32_t K, M, N, r;       /* split N = K*M and number of primes */
    int64_t Y, Y1, Y2;        /* y-transform length Y = Y1*Y2 >= nc */
    int32_t S;                /* middle-pass column slice */
    int64_t Y1b;              /* outer split of Y1 (1 = none) */
    uint32_t primes[8];       /* p_0 > p_1 > ... (r used) */
    double log2_modulus;      /* log2(prod p) */
    double log2_bound;        /* log2(4H), H = min(na,nb)*K*2^(2M-2) */
    size_t workspace_bytes;   /* device bytes the plan allocates */
    int32_t kron;             /* Kronecker packing factor (1 = none); when > 1,
                                 K, M, r, Y... describe the packed product */
    int32_t kron_w;           /* slot width in bits (0 when kron = 1) */
    int64_t kron_na, kron_nb; /* packed coefficient counts */
    uint32_t kron_bits_a, kron_bits_b;  /* packed bit bounds */
    int32_t school;           /* 1: schoolbook family (K, M, r, Y... are 0) */
    int32_t ks;               /* 1: Kronecker substitution; K, M, r, Y...
                                 describe the product of the digit polynomials */
    int32_t ks_w;             /* limbs per slot (Lc + 3), 0 when ks = 0 */
    int32_t kara;             /* Karatsuba levels (0: not that family) */
    int32_t bigp;             /* 1: big-prime form (K, M, N, Y describe it; r = 1) */
} ipm_plan_info;

/*
 * Host-only planner (DetermineBase and RecoveryPrime, §2 and §2.1; the
 * prime-product form of §4).  Touches no GPU.  `params` may be NULL.
 * Returns IPM_ERR_ARG for an invalid shape or override and
 * IPM_ERR_UNSUPPORTED when no plan meets the bounds.
 */
ipm_status ipm_choose(const ipm_shape *shape, const ipm_params *params, ipm_plan_info *out);

/*
 * Create a plan for n product shapes on the current CUDA device: runs the
 * planner, builds the twiddle/CRT tables and allocates the workspace.
 * n = 1 for ipm_mul; n >= 1 for ipm_mul_batched (the i-th operand set of a
 * batched call must match shapes[i]).  `params` (may be NULL) applies to
 * every shape.  On success *out receives the plan; on failure *out = NULL.
 */
ipm_status ipm_plan(ipm_plan_t *out, const ipm_shape *shapes, int32_t n, uint32_t flags);
ipm_status ipm_plan_ex(ipm_plan_t *out, const ipm_shape *shapes, int32_t n, uint32_t flags,
                       const ipm_params *params);

/*
 * Candidate plans of one shape for autotuning and cost-model dispatch: every
 * digit split K from half to eight times the planner's that meets the
 * bounds, with the planner's tiles for it and the tile variants Y2/2, 2 Y2,
 * 4 Y2, S/2 and 2 S (where valid), each as the override set
 * that selects it, the plan it yields, and IPM_FEATURES numbers describing
 * it (log2 of na, nb, bits_a, bits_b, K, Y, Y2, S, Y1b, transform points
 * r*Y*2K, middle column length and total input bits; M/32, r, two kernel
 * variant flags; log2 of the Kronecker packing factor; a schoolbook flag;
 * and log2 of the batch size capped at 16, which is 0 here: the learned
 * dispatch sets it to log2(min(n, 16)) for a plan of n shapes; for the
 * schoolbook family the transform fields are 0 and the points feature is
 * log2 of na nb La Lb).  Candidates with kron > 1 are listed when the slot
 * width allows it (w <= 128), each factor with the planner's plan of the
 * packed product and its K halved and doubled; the schoolbook candidate
 * when its limits allow it.
 * Writes at most `max` entries and returns how many exist (negative status
 * on an invalid shape).
 */
#define IPM_FEATURES 19
typedef struct {
    ipm_params params;
    ipm_plan_info info;
    float features[IPM_FEATURES];
} ipm_candidate;
int32_t ipm_candidates(const ipm_shape *shape, ipm_candidate *out, int32_t max);

/*
 * Learned plan dispatch (no counterpart in the paper, whose DetermineBase,
 * §2.4, reads the split from a precomputed table).  A multilayer perceptron
 * IPM_FEATURES -> 32 -> 32 -> 1 with ReLU maps a candidate's features to
 * its predicted run time.  With the plan flag IPM_COSTMODEL (and params
 * NULL), ipm_plan / ipm_plan_ex take for each shape (1) the measured best
 * plan from the tuning table (ipm_set_tuned) when the shape is in it, else
 * (2) the candidate with the smallest predicted time under the installed
 * model (ipm_set_cost_model), else (3) the analytic planner.  Every
 * candidate computes the same exact product: the model chooses speed only.
 *
 * Model: IPM_MLP_FLOATS host floats: feature means [F], inverse standard
 * deviations [F] (0 for a constant feature), target mean, target standard
 * deviation, then the IPM_MLP_PARAMS parameters W1[32][F], b1[32],
 * W2[32][32], b2[32], w3[32], b3 (F = IPM_FEATURES, row-major).  The network
 * sees standardised features and predicts the standardised target.
 *
 * ipm_mlp_train: n >= 2 host samples X[n][F] (row-major) with targets y[n]:
 *   computes the standardisation, draws Glorot-uniform weights from `seed`
 *   (splitmix64; biases zero), runs `epochs` full-batch Adam steps
 *   (learning rate lr, beta1 0.9, beta2 0.999, on the mean loss) on the GPU
 *   and writes the model to `model`, and the final mean of 1/2 (o - t)^2
 *   to *final_loss (may be NULL).
 * ipm_mlp_grad: for a host model, the sum over samples of 1/2 (o - t)^2
 *   (*loss) and its gradient with respect to the IPM_MLP_PARAMS parameters
 *   (grad[], host), from the GPU kernel that training uses.
 * ipm_mlp_predict: out[i] = the model's prediction for X[i], in target
 *   units (host arrays; n may be 0).
 * ipm_set_cost_model: copy `model` (nfloats = IPM_MLP_FLOATS) for
 *   IPM_COSTMODEL; NULL uninstalls it.
 * ipm_set_tuned: replace the tuning table by n (shape, params) pairs
 *   (n = 0 clears it); if a pair does not plan, its status is returned and
 *   the table is left unchanged.
 * ipm_dispatch: the params IPM_COSTMODEL gives `shape` (all zero: the
 *   analytic planner) and their source (*source: 0 planner, 1 table,
 *   2 model; may be NULL).
 * These run on the current device, allocate their own scratch and wait for
 * it: not for use during stream capture.  Float sums in the gradient are
 * unordered, so trained weights may differ in their last bits between runs.
 */
#define IPM_MLP_HIDDEN 32
#define IPM_MLP_PARAMS \
    (IPM_MLP_HIDDEN * IPM_FEATURES + IPM_MLP_HIDDEN * IPM_MLP_HIDDEN + 3 * IPM_MLP_HIDDEN + 1)
#define IPM_MLP_FLOATS (2 * IPM_FEATURES + 2 + IPM_MLP_PARAMS)
ipm_status ipm_mlp_train(const float *X, const float *y, int32_t n, int32_t epochs, float lr,
                         uint64_t seed, float *model, float *final_loss);
ipm_status ipm_mlp_grad(const float *model, const float *X, const float *y, int32_t n,
                        float *grad, float *loss);
ipm_status ipm_mlp_predict(const float *model, const float *X, int32_t n, float *out);
ipm_status ipm_set_cost_model(const float *model, int32_t nfloats);
ipm_status ipm_set_tuned(const ipm_shape *shapes, const ipm_params *params, int32_t n);
ipm_status ipm_dispatch(const ipm_shape *shape, ipm_params *out, int32_t *source);

/* Plan parameters of shape `index` of a plan. */
ipm_status ipm_get_info(ipm_plan_t plan, int32_t index, ipm_plan_info *out);

/*
 * c = a*b (§2.3, the main algorithm) for a plan with n = 1.
 * a, a_neg, b, b_neg, c, c_neg are DEVICE pointers in the format above,
 * 16-byte aligned for the limb arrays.  c must not overlap a or b.
 */
ipm_status ipm_mul(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg,
                   const uint32_t *b, const uint8_t *b_neg,
                   uint32_t *c, uint8_t *c_neg, ipm_stream_t stream);

/*
 * Same product with HOST buffers (pinned memory is fastest): copies a and b
 * to plan-owned device buffers, multiplies, copies c back and waits for the
 * stream.  The device buffers are allocated on first use and kept.
 */
ipm_status ipm_mul_host(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg,
                        const uint32_t *b, const uint8_t *b_neg,
                        uint32_t *c, uint8_t *c_neg, ipm_stream_t stream);

/*
 * ipm_mul_host without the wait: the copies in, the product and the copies
 * out are enqueued on `stream` and the call returns.  The result is in c
 * and c_neg, and device errors are reported, after ipm_sync(plan, stream).
 * The host buffers must stay valid until then and should be pinned (copies
 * from pageable memory are not asynchronous).  Calls on one plan share its
 * device buffers, so they must be ordered on one stream; a caller overlaps
 * the copies of some products with the compute of others by using several
 * plans on as many streams (three products in flight reach 99% of the
 * device-resident rate for two degree-32767 polynomials of 4096 bits on a
 * GB300; two reach 90%).
 */
ipm_status ipm_mul_host_async(ipm_plan_t plan, const uint32_t *a, const uint8_t *a_neg,
                              const uint32_t *b, const uint8_t *b_neg,
                              uint32_t *c, uint8_t *c_neg, ipm_stream_t stream);

/* Device pointers of one product of a batch (layout as for ipm_mul). */
typedef struct {
    const uint32_t *a;
    const uint8_t *a_neg;
    const uint32_t *b;
    const uint8_t *b_neg;
    uint32_t *c;
    uint8_t *c_neg;
} ipm_operands;

/*
 * n independent products ops[i] with shapes[i] of the plan (n must equal
 * the plan's shape count).  `ops` is a HOST array of device pointers; it may
 * be reused as soon as the call returns.  The plan groups its shapes by
 * kernel variant (at most 4 GiB of workspace per group) and runs each
 * group's products together: three launches per group, every block finding
 * its product and tile in device tables built by ipm_plan.  Products whose
 * plan splits the middle transform, packs coefficients or uses the
 * schoolbook family are launched one by one after the groups.
 * With IPM_GRAPH, the first call records the grouped launches into a CUDA
 * graph (on a stream the plan owns; the kernels read all operand pointers
 * from the plan's device table, which every call refreshes first) and every
 * call launches that graph: one launch for all groups.
 * With IPM_PERSISTENT, the transform and schoolbook products run instead as
 * ONE persistent launch (two 256-thread blocks per SM when every tile fits
 * 112 KB of shared memory, else one 512-thread block) over a device work
 * queue of (product, phase, tile) items: each product in its own workspace
 * slice (the plan allocates all of them: the sum of the products'
 * workspaces), items ordered as a three-stage pipeline over windows of
 * products, every item after the previous phase of its product, which the
 * block awaits with a bounded device wait (ipm_set_wait_limit; a wait that
 * runs out makes the call report IPM_ERR_TIMEOUT).  With IPM_GRAPH too,
 * that launch is the graph.  Products that split the middle transform,
 * pack coefficients or use another family still run one by one after it.
 * A plan whose largest tile leaves no room in one block's shared memory
 * for the persistent kernel keeps the grouped launches.
 */
ipm_status ipm_mul_batched(ipm_plan_t plan, const ipm_operands *ops, int32_t n,
                           ipm_stream_t stream);

/*
 * A product that allocates nothing (no counterpart in the paper; this is an
 * interface convenience).  For callers that cannot allocate device memory
 * while they run: services with latency limits that forbid allocator calls
 * (cudaMalloc may synchronise the device and take milliseconds), and
 * plugins whose host application owns all memory and hands over only the
 * operand and output buffers.
 *
 * Same arguments and layouts as ipm_mul (device pointers), but no plan: the
 * shape is given directly and the planner's default choices are used.  c
 * must hold (deg_a + deg_b + 1) rows of
 *     Lc = ceil((bits_a + bits_b + ceil(log2 min(deg_a + 1, deg_b + 1))) / 32)
 * limbs (the stride ipm_plan_info.lc reports); the library cannot check the
 * size of a raw pointer's buffer, and a smaller c is written past its end.
 * The product's scratch -- error word, twiddle tables and transform
 * workspace -- lives in one static device array of IPM_NOALLOC_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits;
 * products whose scratch does not fit return IPM_ERR_UNSUPPORTED (for
 * example two degree-1023 polynomials with 255-bit coefficients need 0.85
 * MiB, two of degree 2047 with 2048-bit coefficients 12.2 MiB, two of
 * degree 4095 with 4096-bit coefficients 48.4 MiB, which is rejected).
 *
 * The first call on a device looks up the array's device address and sets
 * kernel limits: make it before any stream capture.  All calls share the
 * array, which keeps the previous call's contents (the error word is
 * cleared and the tables rewritten each call).  Calls are serialised by a
 * host lock and each one waits for its `stream` before it returns, so two
 * calls never overlap on the GPU; what can still race is the caller's own
 * work on other streams that touches c while a call runs.  Returns the
 * product's status (IPM_ERR_BOUND for an input above its bit bound).
 */
#define IPM_NOALLOC_SCRATCH_BYTES (32u << 20)
ipm_status ipm_mul_noalloc(const ipm_shape *shape, const uint32_t *a, const uint8_t *a_neg,
                           const uint32_t *b, const uint8_t *b_neg,
                           uint32_t *c, uint8_t *c_neg, ipm_stream_t stream);

/*
 * Randomised check of a finished product (no counterpart in the paper):
 * evaluates a, b and c at one point t derived from `seed` modulo the
 * Mersenne prime q = 2^61 - 1 on the GPU and compares c(t) with a(t) b(t).
 * The exact product always passes.  A wrong c is caught with probability at
 * least 1 - deg(c) / q > 1 - 2^-40 whenever the error polynomial c - a*b is
 * non-zero modulo q (Schwartz-Zippel: a non-zero polynomial of degree D
 * has at most D roots); any single changed limb or sign is such an error.
 * An error that is 0 modulo q (e.g. a sign flipped on a coefficient whose
 * magnitude is a multiple of q) is never caught.  Layouts as in ipm_mul for `shape` (device
 * pointers).  Waits for `stream`; returns IPM_OK or IPM_ERR_MISMATCH.
 * Allocates and frees a few KB of device memory per call.
 */
ipm_status ipm_validate(const ipm_shape *shape, const uint32_t *a, const uint8_t *a_neg,
                        const uint32_t *b, const uint8_t *b_neg,
                        const uint32_t *c, const uint8_t *c_neg, uint64_t seed, ipm_stream_t stream);

/* Wait for `stream`, then return and clear the plan's device error word. */
ipm_status ipm_sync(ipm_plan_t plan, ipm_stream_t stream);

/*
 * IPM_PERSISTENT batched plans (no counterpart in the paper): limit of every
 * device-side dependency wait of the persistent launch, in microseconds
 * (default 2 s, at most 600 s).  A wait that runs out sets IPM_ERR_TIMEOUT
 * (returned by ipm_sync or by an IPM_SYNC call) and the launch returns;
 * the outputs of that call are then incomplete.  IPM_ERR_UNSUPPORTED for a
 * plan without the persistent launch.
 */
ipm_status ipm_set_wait_limit(ipm_plan_t plan, uint64_t microseconds);

/*
 * Test hook for the timeout path of IPM_PERSISTENT plans: from the next
 * batched call on, product `product`'s forward phase counts one tile more
 * than exists, so its later tiles wait until the limit runs out (a
 * condition nothing satisfies); -1 removes the hold.  IPM_ERR_ARG for a
 * product the persistent kernel does not run.
 */
ipm_status ipm_debug_hold(ipm_plan_t plan, int32_t product);

/*
 * Taylor shift by one: g(x) = f(x + 1), exactly, for f of degree `deg`
 * with |f_i| < 2^bits -- the operation the paper's application (§1, real
 * root isolation) builds on its product, there by the divide-and-conquer
 * method (Algorithm E of von zur Gathen and Gerhard, ISSAC 1997).  Here:
 * f padded to n' = 2^m coefficients; at level l (blocks of b = 2^l,
 * already shifted) every pair of blocks (lo, hi) becomes lo + (x+1)^b hi,
 * all pairs of a level in ONE ipm_mul of (x+1)^b by the hi blocks placed
 * 2b apart; (x+1)^b is the square of (x+1)^(b/2) (ipm_mul), all of them
 * computed once by ipm_taylor_plan (which therefore runs work on the GPU
 * and waits for it); the first six levels run in shared memory with
 * additions only; the block additions are sign-magnitude additions on the
 * GPU.
 *
 * Layout: f and g as in ipm_mul (device pointers, sign-magnitude 32-bit
 * limbs); f has stride ceil(bits/32), g has deg+1 coefficients with stride
 * ipm_taylor_limbs() = ceil((bits + deg + 1)/32), since |g_k| <
 * 2^(bits + deg + 1).  The plan owns its buffers and one ipm plan per level
 * (flags IPM_COSTMODEL and IPM_TENSOR_STAGES pass to them; IPM_SYNC makes
 * ipm_taylor_shift wait and return the device status).  Limits:
 * deg < 2^20 and bits + 2^(m-1) <= 65536 (IPM_ERR_UNSUPPORTED).  Device
 * errors (an input above its bound, IPM_ERR_BOUND; an internal bound
 * violation, IPM_ERR_CUDA) are returned by ipm_taylor_sync.
 */
typedef struct ipm_taylor_s *ipm_taylor_t;
ipm_status ipm_taylor_plan(ipm_taylor_t *out, int64_t deg, uint32_t bits, uint32_t flags);
ipm_status ipm_taylor_limbs(ipm_taylor_t t, int32_t *limbs);
ipm_status ipm_taylor_shift(ipm_taylor_t t, const uint32_t *f, const uint8_t *f_neg,
                            uint32_t *g, uint8_t *g_neg, ipm_stream_t stream);
ipm_status ipm_taylor_sync(ipm_taylor_t t, ipm_stream_t stream);
ipm_status ipm_taylor_destroy(ipm_taylor_t t);

/* Free a plan (waits for the device first).  NULL is accepted. */
ipm_status ipm_destroy(ipm_plan_t plan);

/*
 * Per-pass timing.  With profiling enabled, every product a plan runs
 * records CUDA events on its stream before the first pass and after each of
 * the three passes (split + forward transforms; middle transforms +
 * pointwise product; inverse transforms + CRT + recombination).  No work is
 * skipped or reordered.  ipm_phase_ms waits for the events of the most
 * recent product and writes min(n, 3) durations in milliseconds to ms[].
 * ipm_phase_ms returns IPM_ERR_ARG when profiling is off or nothing ran.
 */
ipm_status ipm_set_profiling(ipm_plan_t plan, int32_t enable);
ipm_status ipm_phase_ms(ipm_plan_t plan, float *ms, int32_t n);

/* Static description of a status code. */
const char *ipm_strerror(ipm_status status);

/* Number of kernels this library has launched in this process. */
int64_t ipm_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* IPM_H */
