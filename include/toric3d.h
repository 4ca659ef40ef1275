/*
 * toric3d.h -- C ABI of the GB300 (sm_103a) library for Monte Carlo decoding of
 * the 3D toric code with flip, p-flip and belief propagation, after Scruby &
 * Nemoto, "Local Probabilistic Decoding of a Quantum Code" (arXiv:2212.06985).
 *
 * Conventions shared by every call
 * ---------------------------------
 * Lattice (Sec. 2): periodic L x L x L cubic lattice, qubits on the 3L^3
 * edges, Z checks on the 3L^3 faces (primal picture; the paper draws the
 * equivalent dual one).  Index layout:
 *     edge (d, x, y, z) -> ((d*L + z)*L + y)*L + x        d = edge direction
 *     face (n, x, y, z) -> ((n*L + z)*L + y)*L + x        n = face normal
 * The face with normal n at r is spanned by the two axes a < b other than n
 * and holds the a-edges at r and r+e_b and the b-edges at r and r+e_a.
 *
 * Bit-sliced state: an error or syndrome array is uint64_t[3L^3][words];
 * sample 64*w + j of a batch is bit j of word w.  Lanes past the last sample of
 * the final word are scratch: calls may change them and never report them.
 *
 * Memory: every pointer is a device pointer owned by the caller unless stated
 * otherwise; the library allocates no device memory.  Arrays of uint64_t must
 * be 8-byte aligned, float arrays and workspaces 16-byte aligned.
 *
 * Streams: every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 * legacy default stream) and returns once its kernels are enqueued.
 *
 * Errors: a call returns T3D_OK or an error code and launches nothing when its
 * arguments are invalid (T3D_EINVAL).  T3D_ECUDA reports a CUDA runtime error
 * seen while enqueuing.  toric3d_last_error() returns a message describing the
 * calling thread's last failure.  No exception crosses the ABI.
 *
 * Random numbers (the paper only says "random number in (0,1)", Sec. 3.2):
 * Philox4x32-10 (Salmon et al., SC'11) with key (seed mod 2^32, seed >> 32)
 * and counter (group mod 2^32, site, cycle, stream<<30 | sweep<<8 | block),
 * group = sample / 64; sweep indices stay below 2^22.  Word i (64 bits) of a
 * stream position is outputs 0 | 1<<32 (i even) or 2 | 3<<32 (i odd) of block
 * i/2.  Bernoulli(p) for a sample in lane j is U < P, P = floor(p*2^32 + 1/2),
 * for a 32-bit uniform U: its six high bits (bit 31-i = bit j of word i,
 * i = 0..5) decide the lanes whose six high bits differ from P's; the k-th
 * lane of the 64 (in lane order) whose six high bits equal P's takes its
 * low 26 bits from the high 26 bits of output k%4 of block 3 + k/4.
 * Streams: 0 qubit flips (site = edge), 1 measurement flips (site =
 * face), 2 p-flip coins (site = lattice site r: the coin of r's d-edge is bit
 * j of word d).  `sample0` (a multiple of 64) is the global index of a
 * batch's first sample, so disjoint sample ranges on different GPUs or in
 * resumed runs draw exactly the numbers one large batch would.
 */
#ifndef TORIC3D_H
#define TORIC3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    T3D_OK = 0,
    T3D_EINVAL = 1,     /* invalid argument; nothing was launched */
    T3D_ECUDA = 2,      /* CUDA runtime error while enqueuing work */
    T3D_ETIMEOUT = 3,   /* a bounded device-side wait gave up */
    T3D_EINTERNAL = 4   /* internal consistency check failed */
} t3d_status;

typedef void* t3d_stream; /* cudaStream_t */

/* Message describing the calling thread's most recent failure ("" if none). */
const char* toric3d_last_error(void);

/* ABI revision of this header. */
int toric3d_abi_version(void);

/*
 * Phenomenological qubit noise (Sec. 3.1, Fig. 2 caption): for every edge and
 * every sample of the batch, e ^= Bernoulli(p), drawn from stream 0 at
 * (site = edge, cycle, sweep = 0).  e: uint64_t[3L^3][words], in place.
 * 2 <= L <= 256, words >= 1, 0 <= p <= 1.
 */
t3d_status toric3d_noise(int L, int64_t words, uint64_t* e, double p, uint64_t seed,
                         uint64_t sample0, uint32_t cycle, t3d_stream stream);

/*
 * One noisy syndrome measurement (Sec. 2, Sec. 3.1): s_f = XOR of the four
 * edges of face f, then s ^= Bernoulli(q) from stream 1 at (site = face,
 * cycle).  q = 0 gives the noiseless syndrome H e.  e is read, s overwritten;
 * both uint64_t[3L^3][words] and must not overlap.
 */
t3d_status toric3d_syndrome(int L, int64_t words, const uint64_t* e, uint64_t* s, double q,
                            uint64_t seed, uint64_t sample0, uint32_t cycle,
                            t3d_stream stream);

/* Workspace for toric3d_flip / toric3d_pflip: one bit-sliced syndrome array. */
size_t toric3d_flip_workspace_bytes(int L, int64_t words);

/*
 * Parallel flip (Sec. 3.1 rule; Sec. 3.2 on the parallel version): `sweeps`
 * synchronous applications; in each, every qubit with more unsatisfied than
 * satisfied checks (3 or 4 of its 4 faces) flips, all deciding from the same
 * syndrome snapshot, and the syndrome is updated by the flips (s ^= H f).
 * e and s in place.  work: >= toric3d_flip_workspace_bytes(L, words) bytes of
 * device scratch whose contents are not preserved.
 */
t3d_status toric3d_flip(int L, int64_t words, uint64_t* e, uint64_t* s, int sweeps, void* work,
                        size_t work_bytes, t3d_stream stream);

/* Workspace for toric3d_flip_until_clear: the syndrome copy of toric3d_flip plus
 * 256 bytes of flags. */
size_t toric3d_flip_until_clear_workspace_bytes(int L, int64_t words);

/*
 * Parallel flip until the syndrome clears (Sec. 3.1: the decoder repeats the
 * flip until no check is unsatisfied or a sweep limit is reached): at most
 * max_sweeps applications of the toric3d_flip rule; once an application
 * leaves no unsatisfied check anywhere in the batch, the remaining ones do no
 * work (each checks a device flag at its start, so nothing waits on the host
 * and the call can be captured in a CUDA graph).  The results equal those of
 * toric3d_flip with max_sweeps sweeps: a sample whose syndrome is clear flips
 * nothing.  sweeps_done (device int32, nullable) receives the number of
 * applications that ran from a syndrome with an unsatisfied check: 0 for a
 * clear input, max_sweeps when the batch never clears.  work: >=
 * toric3d_flip_until_clear_workspace_bytes(L, words) bytes, 16-byte aligned,
 * contents not preserved.  0 <= max_sweeps <= 2^22.
 */
t3d_status toric3d_flip_until_clear(int L, int64_t words, uint64_t* e, uint64_t* s, int max_sweeps,
                                    int32_t* sweeps_done, void* work, size_t work_bytes,
                                    t3d_stream stream);

/*
 * toric3d_flip without a workspace argument, for callers that cannot give the
 * library device memory: a decoder in a control loop whose device memory is
 * fixed at start-up, a plugin whose host application owns every device
 * allocation, or a latency-critical caller that cannot risk the device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  The paper has no
 * counterpart; it is the same computation as toric3d_flip.  The scratch
 * syndrome copy lives in a 32 MiB array inside the library (held on every GPU
 * that loads the library until the process exits), so this call allocates
 * nothing.  It rejects (T3D_EINVAL) any L, words with 3 L^3 * words * 8 bytes
 * above 32 MiB.  The first call on a device looks up the array's address with
 * that device current, and so does the first call after the device's CUDA
 * context changed (cudaDeviceReset); make those calls before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race, so
 * order them.  Nothing in the array needs clearing between calls.
 */
t3d_status toric3d_flip_noalloc(int L, int64_t words, uint64_t* e, uint64_t* s, int sweeps,
                                t3d_stream stream);

/*
 * flip + p-flip on a schedule (Sec. 3.2 p-flip rule and schedule list,
 * Table 1 footnote, Sec. 4.2): n_apply synchronous applications whose kinds
 * cycle through `schedule`, a host string over {'F','P'} of length 1..63.  A
 * 'P' application also flips each qubit with exactly 2 of 4 unsatisfied checks
 * whose coin is 1; application k uses coin sweep index sweep0 + k (sweep0 +
 * n_apply <= 2^22).  e and s in place; work as for toric3d_flip.
 */
t3d_status toric3d_pflip(int L, int64_t words, uint64_t* e, uint64_t* s, const char* schedule,
                         int n_apply, uint32_t sweep0, uint64_t seed, uint64_t sample0,
                         uint32_t cycle, void* work, size_t work_bytes, t3d_stream stream);

/*
 * Belief propagation messages.  Samples are processed in rows of 64, the
 * samples of one bit-sliced word.  A message buffer for n samples is
 * float[ceil(n/64)][L^3][3][4][64]: entry (w, site, d, k, i) is the
 * check->variable message M_{f->v} for sample 64w + i into edge v = (d, site)
 * from its k-th face.
 * For an edge along axis a at r, with c0 < c1 the two other axes, its faces
 * are k = 0: normal 3-a-c0 at r; k = 1: that face at r - e_c0; k = 2: normal
 * 3-a-c1 at r; k = 3: that face at r - e_c1.
 */
size_t toric3d_bp_message_bytes(int L, int64_t n_samples);

/*
 * One flooding BP iteration (Sec. 4.1, Eqs. 2-3): from the check->variable
 * messages msg_in (NULL: the first iteration, every variable->check message
 * equal to the prior l0 = log((1-p)/p), Eq. 1) compute every
 * variable->check message l0 + sum of the other three incoming messages
 * (Eq. 3) and from those every new check->variable message
 * (-1)^{s_f} 2 atanh(tq * prod of tanh(m/2) over the other three edges)
 * (Eq. 2), clamped to |M| <= 30, into msg_out.  tq = tanh(lq/2) with
 * lq = log((1-q_meas)/q_meas) is the message of the measurement-error
 * variable attached to each check (Sec. 4.1); q_meas = 0 leaves them out.
 * s: uint64_t[3L^3][ceil(n_samples/64)].  FP32 arithmetic.  msg_in and
 * msg_out must not overlap.
 */
t3d_status toric3d_bp_step(int L, int64_t n_samples, const uint64_t* s, double p, double q_meas,
                           const float* msg_in, float* msg_out, t3d_stream stream);

/*
 * BP hard decision (Sec. 4.1, after Eq. 4): posterior l_v = l0 + sum of the
 * four incoming messages (msg NULL: l_v = l0); every qubit with l_v < 0 is
 * corrected, e ^= d and s ^= H d, in samples 0 .. n_samples - 1 only (the
 * unused tail lanes of the last word get no correction).  llr_out (nullable)
 * receives l_v as
 * float[3L^3][n_samples].  work: >= toric3d_bp_decide_workspace_bytes(L,
 * n_samples) bytes of 32-byte aligned device scratch for the decision words.
 */
size_t toric3d_bp_decide_workspace_bytes(int L, int64_t n_samples);
t3d_status toric3d_bp_decide(int L, int64_t n_samples, const float* msg, double p, uint64_t* e,
                             uint64_t* s, float* llr_out, void* work, size_t work_bytes,
                             t3d_stream stream);

/* Workspace for toric3d_bp processing `chunk_samples` samples at a time. */
size_t toric3d_bp_workspace_bytes(int L, int64_t chunk_samples);

/*
 * Local BP decoder (Sec. 4.1): `iters` flooding iterations from the priors,
 * then the hard decision applied to e and s.  Samples are processed in chunks
 * of whole 64-sample words, as large as the workspace allows (at least one
 * word must fit; see toric3d_bp_workspace_bytes).  llr_out as for
 * toric3d_bp_decide; it needs a workspace for the whole batch.
 */
t3d_status toric3d_bp(int L, int64_t n_samples, uint64_t* e, uint64_t* s, double p,
                      double q_meas, int iters, void* work, size_t work_bytes, float* llr_out,
                      t3d_stream stream);

/*
 * BP with meta-checks (Sec. 4.1, last paragraph, where the paper proposes
 * them without simulating them): every error-free syndrome is a set of closed
 * loops, so the six faces of every unit cube have even parity.  The factor
 * graph has the 3L^3 qubit variables (prior log((1-p)/p)), one measurement-
 * error variable per face (prior log((1-q)/q)) joined to its face check and
 * to the meta-checks of the two cubes the face bounds, the 3L^3 face checks
 * (syndrome s) and the L^3 cube meta-checks (syndrome: parity of s over the
 * cube's six faces).  `iters` flooding iterations of Eqs. 2-3 over that
 * graph from the priors, FP32 messages clamped to |M| <= 30; then every qubit
 * with posterior (Eq. 4) below zero is corrected, e ^= d and s ^= H d.
 *   e, s      uint64_t[3L^3][ceil(n_samples/64)], device, updated in place
 *   0 < p < 1, 0 < q < 1 (q = 0 has no measurement variables: toric3d_bp)
 *   work      >= toric3d_bp_meta_workspace_bytes(L, 64) bytes of 256-byte
 *             aligned device scratch; samples are processed in chunks of
 *             whole 64-sample words as large as it allows
 *   llr_out   nullable: float[2][3L^3][n_samples], the qubits' posteriors
 *             then the measurement variables' (face order); needs a
 *             workspace for all samples at once
 * Returns T3D_EINVAL (message in toric3d_last_error) on a bad argument or a
 * workspace too small for one word; nothing is launched then.
 */
size_t toric3d_bp_meta_workspace_bytes(int L, int64_t chunk_samples);
t3d_status toric3d_bp_meta(int L, int64_t n_samples, uint64_t* e, uint64_t* s, double p, double q,
                           int iters, void* work, size_t work_bytes, float* llr_out, t3d_stream stream);

/*
 * One flooding iteration of the meta-check BP above, for checking it message
 * by message.  Message buffers are float[7][3L^3][S'], S' = 64 ceil(n_samples
 * / 64) samples innermost: rows 4f + j (j = 0..3) face f -> its j-th edge
 * (the a-edges at r and r + e_b, then the b-edges at r and r + e_a, a < b the
 * face's in-plane axes), row 3L^3 * 4 + f face f -> its measurement
 * variable, row 3L^3 * 5 + f the cube at the face's own site (the face is
 * its lower face) -> that variable, row 3L^3 * 6 + f the cube one step down
 * along the face's normal (upper face) -> that variable.  msg_out gets every
 * check -> variable message computed from msg_in (all zero: the first
 * iteration); the buffers must not overlap; toric3d_bp_meta_message_bytes
 * gives their size and work (16-byte aligned device scratch for the edge
 * totals) needs a seventh of it.
 */
size_t toric3d_bp_meta_message_bytes(int L, int64_t n_samples);
t3d_status toric3d_bp_meta_step(int L, int64_t n_samples, const uint64_t* s, double p, double q,
                                const float* msg_in, float* msg_out, void* work, size_t work_bytes,
                                t3d_stream stream);

/*
 * Decoders on a generic Tanner graph.  Sec. 5 asks whether these local
 * decoders carry over to other LDPC codes; these calls run the same rules on
 * any code given by its checks: noise, noisy measurement, flip / p-flip and
 * BP.  A graph is prepared once into a device blob:
 *   cptr int32[n_checks + 1], cvar int32[cptr[n_checks]]  (HOST arrays, CSR:
 *        check c acts on variables cvar[cptr[c]] .. cvar[cptr[c+1]-1]; no
 *        variable twice in a check; every degree <= 32)
 *   blob >= toric3d_tanner_bytes(n_vars, n_checks, cptr[n_checks]) bytes of
 *        256-byte aligned device memory, owned by the caller, which must
 *        outlive every call that uses the graph
 * toric3d_tanner_prepare validates the lists, builds the variable-side lists
 * on the host and copies everything into the blob synchronously; `out` then
 * describes the graph (device pointers into the blob) and is passed by
 * address to the calls below.  Errors: T3D_EINVAL (message in
 * toric3d_last_error) on bad lists or sizes; nothing is written then.
 */
typedef struct {
    int64_t n_vars;
    int64_t n_checks;
    int64_t n_edges;
    int32_t max_var_degree;
    int32_t max_check_degree;
    const int32_t* cptr;    /* device: check -> first Tanner edge (CSR) */
    const int32_t* cvar;    /* device: Tanner edge -> variable */
    const int32_t* vptr;    /* device: variable -> first entry of vedge / vcheck */
    const int32_t* vedge;   /* device: the Tanner edges of each variable, checks ascending */
    const int32_t* vcheck;  /* device: the check of each of those edges */
} t3d_tanner;

size_t toric3d_tanner_bytes(int64_t n_vars, int64_t n_checks, int64_t n_edges);
t3d_status toric3d_tanner_prepare(int64_t n_vars, int64_t n_checks, const int32_t* cptr, const int32_t* cvar,
                                  void* blob, size_t blob_bytes, t3d_tanner* out);

/*
 * Bit-sliced state as on the toric code: e uint64_t[n_vars][W], s
 * uint64_t[n_checks][W], W = ceil(n_samples / 64), sample 64 w + j in bit j
 * of word w; sample0 (a multiple of 64) is the index of the first sample.
 * Noise (Sec. 3.1): e ^= Bernoulli(p) keyed by the variable index (stream 0).
 * Syndrome: s = H e ^ Bernoulli(q) keyed by the check index (stream 1).
 * Generator and keys as in toric3d_noise / toric3d_syndrome, so on the toric
 * code's own graph these equal those calls.  Logical readout of a generic
 * code is the same parity computation: prepare a second graph whose rows are
 * the code's logical Z operators and call toric3d_tanner_syndrome on it with
 * q = 0; bit l of sample i is then the parity of e over logical l.
 */
t3d_status toric3d_tanner_noise(const t3d_tanner* g, int64_t n_samples, uint64_t* e, double p, uint64_t seed,
                                uint64_t sample0, uint32_t cycle, t3d_stream stream);
t3d_status toric3d_tanner_syndrome(const t3d_tanner* g, int64_t n_samples, const uint64_t* e, uint64_t* s,
                                   double q, uint64_t seed, uint64_t sample0, uint32_t cycle, t3d_stream stream);

/*
 * n_apply parallel applications cycling through `schedule` ('F' flip, 'P'
 * p-flip): every variable counts its unsatisfied checks u in the current
 * syndrome; it flips when u > deg - u (Sec. 3.1) and, in p-flip, when
 * u == deg - u and its coin is 1 (Sec. 3.2); then e ^= f and s ^= H f.
 * Application k keys the coins with sweep sweep0 + k (sweep0 + n_apply <=
 * 2^22); the coin of variable v is bit (sample mod 64) of word v mod 4 of
 * stream 2 keyed by site v / 4.  work: toric3d_tanner_flip_workspace_bytes of
 * 8-byte aligned device scratch (the flip words).
 */
size_t toric3d_tanner_flip_workspace_bytes(const t3d_tanner* g, int64_t n_samples);
t3d_status toric3d_tanner_pflip(const t3d_tanner* g, int64_t n_samples, uint64_t* e, uint64_t* s,
                                const char* schedule, int n_apply, uint32_t sweep0, uint64_t seed, uint64_t sample0,
                                uint32_t cycle, void* work, size_t work_bytes, t3d_stream stream);

/*
 * Product-sum BP (Sec. 4.1, Eqs. 1-4) with one prior LLR per variable
 * (prior: device float[n_vars]; measurement errors are modelled by adding
 * variables to the graph): `iters` flooding iterations from the priors, FP32
 * messages clamped to |M| <= 30, then every variable with posterior < 0 is
 * corrected, e ^= d and s ^= H d.  work >= toric3d_tanner_bp_workspace_bytes
 * (g, 64) bytes of 256-byte aligned device scratch; samples run in chunks of
 * whole words as large as it allows.  llr_out (nullable): float[n_vars]
 * [n_samples] posteriors; it needs a workspace for all samples at once.
 * toric3d_tanner_bp_step runs one iteration for message-by-message checks:
 * messages float[n_edges][S'] (S' = 64 W, samples innermost, Tanner edges in
 * the CSR order of cptr / cvar), msg_in all zero for the first iteration,
 * msg_in and msg_out of toric3d_tanner_bp_message_bytes each and not
 * overlapping, work >= n_vars * S' floats (16-byte aligned).
 */
size_t toric3d_tanner_bp_workspace_bytes(const t3d_tanner* g, int64_t chunk_samples);
t3d_status toric3d_tanner_bp(const t3d_tanner* g, int64_t n_samples, uint64_t* e, uint64_t* s, const float* prior,
                             int iters, void* work, size_t work_bytes, float* llr_out, t3d_stream stream);
size_t toric3d_tanner_bp_message_bytes(const t3d_tanner* g, int64_t n_samples);
t3d_status toric3d_tanner_bp_step(const t3d_tanner* g, int64_t n_samples, const uint64_t* s, const float* prior,
                                  const float* msg_in, float* msg_out, void* work, size_t work_bytes,
                                  t3d_stream stream);

/*
 * Fallback gate of the learned pre-decoder (no counterpart in the paper,
 * whose decoders have no fallback): gate[w] = 1 iff some sample of word w has
 * more than max_weight unsatisfied checks in s (s: uint64_t[3L^3][words],
 * gate: uint8_t[words], device).  n_flagged (device, nullable) += the number
 * of flagged words.  work: device scratch of toric3d_gate_workspace_bytes.
 */
size_t toric3d_gate_workspace_bytes(int L, int64_t words);
t3d_status toric3d_gate(int L, int64_t words, const uint64_t* s, uint32_t max_weight, uint8_t* gate,
                        int64_t* n_flagged, void* work, size_t work_bytes, t3d_stream stream);

/*
 * Logical readout (Sec. 3.1 and its footnote, Fig. 2 caption, App. A.2): for
 * each axis d the L^2 straight lines of d-edges are a complete set of
 * disjoint logical Z operators; the number c_d of lines with odd residual
 * parity decides a logical X error on qubit d iff 2 c_d >= L^2 (a tie counts
 * as a failure).  mask: uint8_t[n_samples], bit d = axis d.  counts8
 * (nullable): int64_t[8], overwritten with the number of samples showing each
 * mask value.
 */
t3d_status toric3d_logical(int L, int64_t n_samples, const uint64_t* e, uint8_t* mask,
                           int64_t* counts8, t3d_stream stream);

/*
 * Layout conversion: bits uint8_t[n_samples][n_bits] (one sample per row, 0/1
 * values) <-> words uint64_t[n_bits][ceil(n_samples/64)].  Packing zeroes the
 * unused tail lanes.
 */
t3d_status toric3d_pack(int64_t n_bits, int64_t n_samples, const uint8_t* bits, uint64_t* words,
                        t3d_stream stream);
t3d_status toric3d_unpack(int64_t n_bits, int64_t n_samples, const uint64_t* words,
                          uint8_t* bits, t3d_stream stream);

/*
 * A whole Monte Carlo run (Sec. 3.1 Fig. 2, Sec. 3.2, Sec. 4.2).  For cycles
 * t = cycle0+1 .. cycle0+T: qubit noise (p), one noisy measurement (q),
 * optional BP (bp_iters iterations; bp_meas_nodes 0: checks taken as exact,
 * 1: a measurement-error variable per check, 2: those variables joined by the
 * cube meta-checks as in toric3d_bp_meta) with its hard decision, then n_apply flip/p-flip
 * applications cycling through `schedule` (application k keys the coins with
 * sweep index k).  Optionally a final noiseless measurement (cycle0+T+1)
 * decoded by up to perfect_max_sweeps flip applications, the ones after an
 * item's syndrome clears skipped on the device as in toric3d_flip_until_clear
 * (same results).  Finally the logical readout into mask / counts8.
 */
typedef struct {
    int32_t L;
    int32_t T;
    double p;
    double q;
    uint64_t seed;
    uint64_t sample0;          /* multiple of 64 */
    int64_t n_samples;
    int32_t use_bp;
    int32_t bp_iters;
    int32_t bp_meas_nodes;
    int32_t n_apply;
    char schedule[64];         /* NUL-terminated, over {'F','P'}; may be empty iff n_apply == 0 */
    int32_t perfect_round;
    int32_t perfect_max_sweeps;
    uint32_t cycle0;
    int32_t use_graph;         /* 1: capture the T cycles in a CUDA graph and launch it once */
    int64_t bp_chunk_samples;  /* BP (and pre-decoder) chunk size; 0 = as large as the workspace allows */
    const void* cnn_blob;      /* learned pre-decoder (toric3d_cnn_prepare) decoding in place of BP
                                  (use_bp must be 0; toric3d_run_batch only, items carry s_prev); NULL = none */
    int32_t fallback_max_weight; /* with cnn_blob: after the schedule, every 64-sample word in which a sample
                                    keeps more than this many unsatisfied checks (plus the allowance of
                                    fallback_sigmas) is decoded again from the cycle's start (the error
                                    after the noise, the measured syndrome) by BP (bp_iters) + the
                                    schedule, whose result replaces the learned one; -1 = no fallback */
    double fallback_sigmas;      /* > 0: the threshold of each lattice also allows the unsatisfied checks the
                                    noisy measurement alone leaves, floor(q n + fallback_sigmas sqrt(q (1-q) n))
                                    with n = 3L^3 (isolated measurement errors stay unsatisfied after any
                                    decoder); 0 = none */
} t3d_run_cfg;

/* Workspace toric3d_run_cycles needs for `cfg` (uses cfg->bp_chunk_samples, 0 = all). */
size_t toric3d_run_workspace_bytes(const t3d_run_cfg* cfg);

/*
 * e: uint64_t[3L^3][ceil(n_samples/64)], the error state, read at the start
 * (zero it for a fresh code) and left holding the final residual error, so a
 * run split at any cycle resumes exactly.  mask / counts8 as for
 * toric3d_logical (either may be NULL).  cfg is read on the host during the
 * call only.
 */
t3d_status toric3d_run_cycles(const t3d_run_cfg* cfg, uint64_t* e, void* work, size_t work_bytes,
                              uint8_t* mask, int64_t* counts8, t3d_stream stream);

/*
 * Learned local pre-decoder (not in the paper; it stands in for BP ahead of
 * the flip / p-flip schedule).  A periodic 3-D convolutional network:
 * conv 3x3x3 (6 -> 16) + ReLU, conv 3x3x3 (16 -> 16) + ReLU, conv 3x3x3
 * (16 -> 16) + ReLU, 1x1x1 head (16 -> 3), sigmoid.  The six input channels of
 * site r are s_prev(n, r) and s(n, r) for the face normals n = 0, 1, 2 (0/1);
 * output d of site r is the flip probability of edge (d, r).  Parameters are
 * FP32 in PyTorch order: conv1.weight [16][6][3][3][3], conv1.bias [16],
 * conv2.weight [16][16][3][3][3], conv2.bias, conv3.weight, conv3.bias,
 * head.weight [3][16], head.bias [3] (toric3d_cnn_param_count() = 16,515);
 * kernel index (kz, ky, kx) reads the neighbour at (x+kx-1, y+ky-1, z+kz-1),
 * periodic.  Kernels use BF16 weights and activations with FP32 accumulation
 * on the tensor cores; hidden activations are rounded to BF16 between layers.
 *
 * toric3d_cnn_prepare: params (device FP32) -> blob (toric3d_cnn_blob_bytes(),
 * device, 16-byte aligned) in the kernels' layouts.
 * toric3d_cnn_decode: logits from (s_prev, s), corrections d = [logit > 0]
 * applied as e ^= d and s ^= H d.  logits_out (nullable) receives
 * float[3][L^3][n_samples].  work: toric3d_cnn_workspace_bytes(L, n).
 * toric3d_cnn_train_step: one Adam step (lr > 0) of mean binary cross-entropy
 * between the logits and the labels e_label (bit-sliced, the error before
 * decoding) on this batch; params, adam_m, adam_v (device FP32) are updated in
 * place and blob re-prepared; grads_out (nullable, FP32 [param_count])
 * receives the gradient; loss_out (device float) the summed loss.  lr = 0
 * computes gradient and loss only.  work: toric3d_cnn_train_workspace_bytes.
 */
int toric3d_cnn_param_count(void);
size_t toric3d_cnn_blob_bytes(void);
t3d_status toric3d_cnn_prepare(const float* params, void* blob, t3d_stream stream);
size_t toric3d_cnn_workspace_bytes(int L, int64_t n_samples);
t3d_status toric3d_cnn_decode(int L, int64_t n_samples, const uint64_t* s_prev, uint64_t* s,
                              uint64_t* e, const void* blob, float* logits_out, void* work,
                              size_t work_bytes, t3d_stream stream);
/* T3D_OK, or T3D_ETIMEOUT if a tensor-core pre-decoder kernel gave up one of
 * its bounded waits (its results are then invalid) since the last call.
 * Reads and clears the device flag; synchronises the device. */
t3d_status toric3d_cnn_status(void);
/* Test hook: bound (ns) of the pre-decoder's bounded waits that may give up
 * (default and maximum 1 s; 0 restores the default).  A short bound makes
 * those waits run out, so the give-up path (error flag, wind-down that still
 * waits up to 1 s for the kernel's own copies and MMAs in flight, TMEM freed)
 * can be exercised without a fault.  Synchronises the device; process-wide
 * state of the calling device. */
t3d_status toric3d_cnn_debug_wait_limit(uint64_t ns);
size_t toric3d_cnn_train_workspace_bytes(int L, int64_t n_samples);
t3d_status toric3d_cnn_train_step(int L, int64_t n_samples, const uint64_t* s_prev,
                                  const uint64_t* s, const uint64_t* e_label, float* params,
                                  float* adam_m, float* adam_v, int step, float lr, void* blob,
                                  float* grads_out, float* loss_out, void* work, size_t work_bytes,
                                  t3d_stream stream);

/*
 * Batched runs over lattices of different sizes (measurement support for the
 * paper's multi-size threshold plots, Fig. 2, 6, 7).  Up to 8 independent
 * ensembles, each with its own L, sample range and state, advance through the
 * same cycles with the decoder settings of `cfg` (its L, n_samples and sample0
 * are ignored); every step is one launch over all ensembles.  e,
 * mask and counts8 of each item are as for toric3d_run_cycles.  BP chunks are
 * sized per item so the workspace holds one chunk of every item (rounds are
 * added until it does).
 */
typedef struct {
    int32_t L;
    int64_t n_samples;
    uint64_t sample0;          /* multiple of 64 */
    uint64_t* e;               /* device, uint64_t[3L^3][ceil(n_samples/64)], in/out */
    uint8_t* mask;             /* device, uint8_t[n_samples], nullable */
    int64_t* counts8;          /* device, int64_t[8], nullable */
    uint64_t* s_prev;          /* learned decoder: device, like e, the previous cycle's measured syndrome
                                  (zero for a fresh run), in/out; otherwise unused */
    int64_t* fallback_words;   /* learned decoder: device counter, nullable, += words sent to the fallback */
} t3d_batch_item;

size_t toric3d_run_batch_workspace_bytes(const t3d_run_cfg* cfg, const t3d_batch_item* items,
                                         int n_items);
t3d_status toric3d_run_batch(const t3d_run_cfg* cfg, const t3d_batch_item* items, int n_items,
                             void* work, size_t work_bytes, t3d_stream stream);

/*
 * Launch tuning (not in the paper).  Every run kernel is a persistent
 * grid-stride kernel of SMs x resident blocks; a positive cap limits the
 * resident blocks per SM of one kernel kind (0 restores the occupancy limit).
 * toric3d_autotune_batch() plans `work` exactly as toric3d_run_batch() would,
 * measures one noisy syndrome of the items' states into it (e is only read),
 * times the BP iteration on every item's first chunk under each cap and keeps
 * the fastest for the process; it synchronises `stream`, so call it outside
 * stream capture, before the runs it tunes.  The chosen cap and the time of
 * one iteration are returned through the nullable out pointers.
 */
void toric3d_set_blocks_per_sm(int kind, int blocks_per_sm);
int toric3d_get_blocks_per_sm(int kind);
t3d_status toric3d_autotune_batch(const t3d_run_cfg* cfg, const t3d_batch_item* items, int n_items,
                                  void* work, size_t work_bytes, int* bp_blocks_per_sm, float* bp_ms,
                                  t3d_stream stream);

/*
 * Kernel timing (not in the paper; measurement support).  While enabled, every
 * kernel the library enqueues outside a stream capture is bracketed by a pair
 * of CUDA events on its own stream.  toric3d_profile_read() waits for the
 * recorded events and returns, for one kernel kind, the summed device time in
 * milliseconds and the number of launches; toric3d_profile_reset() forgets
 * them.  Host-side state is global to the process; do not toggle it while
 * another thread is enqueuing toric3d work.
 */
typedef enum {
    T3D_K_NOISE = 0,
    T3D_K_SYNDROME = 1,
    T3D_K_FLIP = 2,
    T3D_K_PFLIP = 3,
    T3D_K_BP_STEP = 4,
    T3D_K_BP_DECIDE = 5,
    T3D_K_LOGICAL = 6,
    T3D_K_LAYOUT = 7,
    T3D_K_CNN = 8,
    T3D_K_COUNT = 9
} t3d_kernel_kind;

void toric3d_profile_enable(int on);
void toric3d_profile_reset(void);
t3d_status toric3d_profile_read(int kind, double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* TORIC3D_H */
