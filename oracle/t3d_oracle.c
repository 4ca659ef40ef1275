/*
 * t3d_oracle.c -- plain, slow, per-sample CPU oracle for the 3D toric code
 * decoders of Scruby & Nemoto, "Local Probabilistic Decoding of a Quantum
 * Code" (arXiv:2212.06985).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is
 * compared against.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA library: every index map, the random generator and the
 * decoders are written here from the paper's definitions.
 *
 * State is one sample at a time, one uint8_t per bit; belief propagation is
 * in IEEE binary64.  Nothing is blocked, fused or reordered beyond what the
 * definitions state.
 *
 * Lattice (Sec. 2): periodic L x L x L cubic lattice, qubits on the 3L^3
 * edges, Z checks on the 3L^3 faces (the primal picture; Sec. 2 describes
 * the equivalent dual one).  Public index layout:
 *     edge (d, x, y, z)  ->  ((d*L + z)*L + y)*L + x      d = edge direction
 *     face (n, x, y, z)  ->  ((n*L + z)*L + y)*L + x      n = face normal
 * The face with normal n at r is spanned by the two axes a < b other than n;
 * its four edges are the a-edges at r and r+e_b and the b-edges at r and
 * r+e_a.
 *
 * Random numbers (the paper only says "random number in (0,1)", Sec. 3.2):
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed mod 2^32,
 * seed >> 32), counter = (group mod 2^32, site, cycle, stream<<30 | sweep<<8
 * | block), where group = sample / 64 (sweep < 2^22).  A block gives two
 * 64-bit words: word i is outputs 2(i%2) (low half) and 2(i%2)+1 (high half)
 * of block i/2.  Bernoulli(p) for a sample with lane = sample % 64, with
 * P = floor(p * 2^32 + 0.5): the event is U < P for a 32-bit uniform U whose
 * six high bits (bit 31-j = bit `lane` of word j, j = 0..5, blocks 0..2)
 * decide it whenever they differ from P's six high bits; the lanes of the
 * group whose six high bits equal P's take U's low 26 bits from one 32-bit
 * block output each -- the k-th such lane in lane order (k = 0, 1, ...) the
 * high 26 bits of output k % 4 of block 3 + k/4 -- and their event is
 * low26(U) < low26(P).  The p-flip coin of
 * the d-edge at site r is bit `lane` of word d of stream 2 keyed by site r
 * (blocks 0 and 1 serve the three edges of a site).
 *
 * Parity pins: Philox against its published known-answer vectors and
 * Triton's independent implementation; syndrome against the
 * code parameters [[3L^3,3,L]] of Sec. 2 (GF(2) rank 2L^3-2, weight-4 rows
 * and columns, zero-syndrome membranes and vertex stabilisers); flip and
 * p-flip against the worked examples of Sec. 3 (Fig. 3(a), 3(b), Fig. 5,
 * the opposite-face pair); BP against exact marginals on acyclic Tanner
 * graphs and the closed form of its first iteration; the logical readout
 * against membranes and stabilisers; the generic Tanner-graph decoders
 * against the toric ones on the toric code's own graph, the stated coin
 * key, and single errors of the 2D toric code (hypergraph product of two
 * cycles).  See tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 from its published definition (SC'11, Sec. 3 of that  */
/* paper): ten rounds of two 32x32->64 multiplies, a fixed permutation  */
/* and a Weyl-sequence key schedule.                                    */
/* ------------------------------------------------------------------ */
void t3o_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mult0 * c0;
        uint64_t prod1 = (uint64_t)mult1 * c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { STREAM_QUBIT = 0, STREAM_MEAS = 1, STREAM_COIN = 2 };

/* Word i (64 bits) of the random stream at (seed, stream, site, cycle, sweep,
 * group): outputs 2(i%2) (low half) and 2(i%2)+1 (high half) of block i/2,
 * counter (group mod 2^32, site, cycle, stream<<30 | sweep<<8 | i/2), key
 * (seed mod 2^32, seed >> 32). */
static uint64_t stream_word(uint64_t seed, int stream, uint64_t site, uint64_t cycle, uint64_t sweep,
                            uint64_t group, int i)
{
    uint32_t ctr[4] = { (uint32_t)group, (uint32_t)site, (uint32_t)cycle,
                        ((uint32_t)stream << 30) | ((uint32_t)sweep << 8) | (uint32_t)(i / 2) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    t3o_philox4x32(ctr, key, out);
    int j = 2 * (i % 2);
    return (uint64_t)out[j] | ((uint64_t)out[j + 1] << 32);
}

uint64_t t3o_prob_to_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ULL << 32;
    return (uint64_t)floor(p * 4294967296.0 + 0.5);
}

/* The six high bits of U for every lane of a group: bit 5-j of lane l's value is bit l
 * of stream word j (j = 0..5). */
static void high6_of_group(uint64_t seed, int stream, uint64_t site, uint64_t cycle, uint64_t sweep,
                           uint64_t group, uint32_t high6[64])
{
    for (int l = 0; l < 64; ++l) high6[l] = 0;
    for (int j = 0; j < 6; ++j) {
        uint64_t w = stream_word(seed, stream, site, cycle, sweep, group, j);
        for (int l = 0; l < 64; ++l) high6[l] |= (uint32_t)((w >> l) & 1ULL) << (5 - j);
    }
}

/* The 26-bit value a lane whose six high bits tie P's takes as U's low bits: the lane is the
 * k-th tied lane of its group (k counts the tied lanes below it), and the value is the high 26
 * bits of output k % 4 of block 3 + k/4 of the stream position. */
static uint32_t tail26(uint64_t seed, int stream, uint64_t site, uint64_t cycle, uint64_t sweep,
                       uint64_t group, int k)
{
    uint32_t ctr[4] = { (uint32_t)group, (uint32_t)site, (uint32_t)cycle,
                        ((uint32_t)stream << 30) | ((uint32_t)sweep << 8) | (uint32_t)(3 + k / 4) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    t3o_philox4x32(ctr, key, out);
    return out[k % 4] >> 6;
}

int t3o_bernoulli(double p, uint64_t seed, int stream, uint64_t site, uint64_t cycle,
                  uint64_t sweep, uint64_t sample)
{
    uint64_t thr = t3o_prob_to_threshold(p);
    if (thr == 0) return 0;
    if (thr >= (1ULL << 32)) return 1;
    uint64_t group = sample / 64;
    int lane = (int)(sample % 64);
    uint32_t high6[64];
    high6_of_group(seed, stream, site, cycle, sweep, group, high6);
    uint32_t p_high = (uint32_t)(thr >> 26), p_low = (uint32_t)(thr & ((1u << 26) - 1));
    if (high6[lane] != p_high) return high6[lane] < p_high;
    int k = 0;
    for (int l = 0; l < lane; ++l) k += high6[l] == p_high;
    return tail26(seed, stream, site, cycle, sweep, group, k) < p_low;
}

/* The events of samples [sample0, sample0 + n) of one stream position (statistical tests). */
int64_t t3o_bernoulli_count(double p, uint64_t seed, int stream, uint64_t site, uint64_t cycle,
                            uint64_t sweep, uint64_t sample0, int64_t n)
{
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) c += t3o_bernoulli(p, seed, stream, site, cycle, sweep, sample0 + (uint64_t)i);
    return c;
}

int t3o_coin(uint64_t seed, uint64_t site, int dir, uint64_t cycle, uint64_t sweep, uint64_t sample)
{
    uint64_t w = stream_word(seed, STREAM_COIN, site, cycle, sweep, sample / 64, dir);
    return (int)((w >> (sample % 64)) & 1ULL);
}

/* ------------------------------------------------------------------ */
/* Lattice incidence (Sec. 2).                                          */
/* ------------------------------------------------------------------ */
static int64_t edge_id(int L, int d, const int r[3])
{
    return (((int64_t)d * L + r[2]) * L + r[1]) * L + r[0];
}

static void face_coords(int L, int64_t f, int* n, int r[3])
{
    r[0] = (int)(f % L);
    r[1] = (int)((f / L) % L);
    r[2] = (int)((f / ((int64_t)L * L)) % L);
    *n = (int)(f / ((int64_t)L * L * L));
}

/* The four edges on the boundary of face f. */
void t3o_face_edges(int L, int64_t f, int64_t out[4])
{
    int n, r[3];
    face_coords(L, f, &n, r);
    int a = (n == 0) ? 1 : 0;          /* the two in-plane axes, a < b */
    int b = (n == 2) ? 1 : 2;
    int r_plus_a[3] = { r[0], r[1], r[2] };
    int r_plus_b[3] = { r[0], r[1], r[2] };
    r_plus_a[a] = (r[a] + 1) % L;
    r_plus_b[b] = (r[b] + 1) % L;
    out[0] = edge_id(L, a, r);
    out[1] = edge_id(L, a, r_plus_b);
    out[2] = edge_id(L, b, r);
    out[3] = edge_id(L, b, r_plus_a);
}

/* Face->edge (4 per face) and edge->face (4 per edge) tables.  The
 * edge->face lists are in ascending face order. */
void t3o_incidence(int L, int32_t* face_edges, int32_t* edge_faces)
{
    int64_t n = 3LL * L * L * L;
    int* fill = (int*)calloc((size_t)n, sizeof(int));
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        t3o_face_edges(L, f, ed);
        for (int j = 0; j < 4; ++j) {
            if (face_edges) face_edges[4 * f + j] = (int32_t)ed[j];
            if (edge_faces) edge_faces[4 * ed[j] + fill[ed[j]]] = (int32_t)f;
            fill[ed[j]]++;
        }
    }
    free(fill);
}

/* Noiseless syndrome s = H e: each face is the XOR of its four edges (Sec. 2). */
void t3o_syndrome(int L, const uint8_t* e, uint8_t* s)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        t3o_face_edges(L, f, ed);
        s[f] = (uint8_t)((e[ed[0]] ^ e[ed[1]] ^ e[ed[2]] ^ e[ed[3]]) & 1);
    }
}

/* ------------------------------------------------------------------ */
/* Phenomenological noise (Sec. 3.1, caption of Fig. 2): per code cycle */
/* each qubit suffers an X flip with probability p and each Z-check     */
/* outcome is flipped with probability q.                               */
/* ------------------------------------------------------------------ */
void t3o_noise(int L, uint8_t* e, double p, uint64_t seed, uint64_t sample, uint32_t cycle)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t v = 0; v < n; ++v)
        if (t3o_bernoulli(p, seed, STREAM_QUBIT, (uint64_t)v, cycle, 0, sample))
            e[v] ^= 1;
}

void t3o_measure(int L, const uint8_t* e, uint8_t* s, double q, uint64_t seed,
                 uint64_t sample, uint32_t cycle)
{
    int64_t n = 3LL * L * L * L;
    t3o_syndrome(L, e, s);
    for (int64_t f = 0; f < n; ++f)
        if (t3o_bernoulli(q, seed, STREAM_MEAS, (uint64_t)f, cycle, 0, sample))
            s[f] ^= 1;
}

/* ------------------------------------------------------------------ */
/* flip and p-flip, parallel version (Sec. 3.1 algorithm, Sec. 3.2      */
/* algorithm, and the parallel/sequential discussion around Fig. 5):    */
/* every qubit decides from the same syndrome snapshot; a qubit with    */
/* more unsatisfied than satisfied checks (3 or 4 of its 4) flips; in   */
/* p-flip a qubit with exactly 2 of 4 unsatisfied flips when its coin   */
/* is 1.  The syndrome is updated by the flips (s ^= H f) so the next   */
/* application sees the decoder's current syndrome.                     */
/* ------------------------------------------------------------------ */
static void apply_rule(int L, uint8_t* e, uint8_t* s, int probabilistic, uint64_t seed,
                       uint64_t sample, uint32_t cycle, uint32_t sweep)
{
    int64_t n = 3LL * L * L * L;
    int32_t* ef = (int32_t*)malloc((size_t)n * 4 * sizeof(int32_t));
    uint8_t* flip = (uint8_t*)calloc((size_t)n, 1);
    t3o_incidence(L, NULL, ef);
    for (int64_t v = 0; v < n; ++v) {
        int unsat = s[ef[4 * v]] + s[ef[4 * v + 1]] + s[ef[4 * v + 2]] + s[ef[4 * v + 3]];
        int sat = 4 - unsat;
        if (sat < unsat)
            flip[v] = 1;
        else if (probabilistic && sat == unsat)
            flip[v] = (uint8_t)t3o_coin(seed, (uint64_t)(v % ((int64_t)L * L * L)), (int)(v / ((int64_t)L * L * L)),
                                        cycle, sweep, sample);
    }
    for (int64_t v = 0; v < n; ++v) {
        if (!flip[v]) continue;
        e[v] ^= 1;
        for (int j = 0; j < 4; ++j) s[ef[4 * v + j]] ^= 1;
    }
    free(flip);
    free(ef);
}

void t3o_flip_once(int L, uint8_t* e, uint8_t* s)
{
    apply_rule(L, e, s, 0, 0, 0, 0, 0);
}

void t3o_pflip_once(int L, uint8_t* e, uint8_t* s, uint64_t seed, uint64_t sample,
                    uint32_t cycle, uint32_t sweep)
{
    apply_rule(L, e, s, 1, seed, sample, cycle, sweep);
}

/* Sequential flip (the Sec. 3.1 algorithm taken literally): while some bit
 * has more unsatisfied than satisfied checks, flip the lowest-indexed such
 * bit.  Returns the number of flips, or -1 if max_flips was reached. */
int t3o_flip_sequential(int L, uint8_t* e, uint8_t* s, int max_flips)
{
    int64_t n = 3LL * L * L * L;
    int32_t* ef = (int32_t*)malloc((size_t)n * 4 * sizeof(int32_t));
    t3o_incidence(L, NULL, ef);
    int flips = 0;
    for (;;) {
        int64_t pick = -1;
        for (int64_t v = 0; v < n && pick < 0; ++v) {
            int unsat = s[ef[4 * v]] + s[ef[4 * v + 1]] + s[ef[4 * v + 2]] + s[ef[4 * v + 3]];
            if (4 - unsat < unsat) pick = v;
        }
        if (pick < 0) break;
        if (flips == max_flips) { flips = -1; break; }
        e[pick] ^= 1;
        for (int j = 0; j < 4; ++j) s[ef[4 * pick + j]] ^= 1;
        flips++;
    }
    free(ef);
    return flips;
}

/* ------------------------------------------------------------------ */
/* Product-sum belief propagation in the log domain (Sec. 4.1, Eqs. 1-4) */
/* on a general Tanner graph given in CSR form: check c owns Tanner     */
/* edges cptr[c] .. cptr[c+1]-1, Tanner edge t joins check c to         */
/* variable cvar[t].  Messages live on Tanner edges.                    */
/*   init:      M_{v->c} = l0                       (Eq. 1 prior)       */
/*   check:     M_{c->v} = (-1)^{s_c} 2 atanh( tq * prod_{v' != v}      */
/*                         tanh(M_{v'->c}/2) )      (Eq. 2)             */
/*   variable:  M_{v->c} = l0 + sum_{c' != c} M_{c'->v}   (Eq. 3)       */
/*   posterior: l_v = l0 + sum_c M_{c->v}           (Eq. 4)             */
/* tq = tanh(lq/2) is the constant message of the degree-1 measurement- */
/* error variable attached to each check (Sec. 4.1, last paragraph);    */
/* lq = +inf gives tq = 1, i.e. no measurement nodes.  Numerical guards */
/* (not in the paper): |atanh argument| <= 1 - 1e-15 and |M_{c->v}| <=  */
/* 30.  If m_in is given, it holds check->variable messages after some  */
/* earlier iteration and the first computed iteration starts from the   */
/* variable->check messages those imply (Eq. 3).                        */
/* ------------------------------------------------------------------ */
void t3o_bp(int nv, int nc, const int32_t* cptr, const int32_t* cvar, const uint8_t* syn,
            double l0, double lq, int iters, const double* m_in, double* m_out, double* llr)
{
    int ne = cptr[nc];
    double* vc = (double*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
    double* cv = (double*)calloc((size_t)(ne > 0 ? ne : 1), sizeof(double));
    double* tv = (double*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
    int* vdeg = (int*)calloc((size_t)nv + 1, sizeof(int));
    int* vptr = (int*)calloc((size_t)nv + 1, sizeof(int));
    int* vedge = (int*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(int));
    const double tq = isinf(lq) ? 1.0 : tanh(lq / 2.0);
    const double cap = 1.0 - 1e-15;

    for (int t = 0; t < ne; ++t) vdeg[cvar[t]]++;
    for (int v = 0; v < nv; ++v) vptr[v + 1] = vptr[v] + vdeg[v];
    memset(vdeg, 0, (size_t)nv * sizeof(int));
    for (int t = 0; t < ne; ++t) {
        int v = cvar[t];
        vedge[vptr[v] + vdeg[v]++] = t;
    }

    int have_cv = 0;
    if (m_in) {
        memcpy(cv, m_in, (size_t)ne * sizeof(double));
        have_cv = 1;
    }
    for (int it = 0; it < iters; ++it) {
        /* variable -> check (Eq. 3), or the prior on the very first pass */
        for (int v = 0; v < nv; ++v) {
            for (int i = vptr[v]; i < vptr[v + 1]; ++i) {
                int t = vedge[i];
                double m = l0;
                if (have_cv)
                    for (int i2 = vptr[v]; i2 < vptr[v + 1]; ++i2)
                        if (i2 != i) m += cv[vedge[i2]];
                vc[t] = m;
            }
        }
        /* check -> variable (Eq. 2) */
        for (int t = 0; t < ne; ++t) tv[t] = tanh(vc[t] / 2.0);
        for (int c = 0; c < nc; ++c) {
            for (int t = cptr[c]; t < cptr[c + 1]; ++t) {
                double prod = tq;
                for (int t2 = cptr[c]; t2 < cptr[c + 1]; ++t2)
                    if (t2 != t) prod *= tv[t2];
                if (prod > cap) prod = cap;
                if (prod < -cap) prod = -cap;
                double m = 2.0 * atanh(prod);
                if (syn[c] & 1) m = -m;
                if (m > 30.0) m = 30.0;
                if (m < -30.0) m = -30.0;
                cv[t] = m;
            }
        }
        have_cv = 1;
    }
    /* posterior (Eq. 4) */
    if (llr) {
        for (int v = 0; v < nv; ++v) {
            double l = l0;
            if (have_cv)
                for (int i = vptr[v]; i < vptr[v + 1]; ++i) l += cv[vedge[i]];
            llr[v] = l;
        }
    }
    if (m_out) memcpy(m_out, cv, (size_t)ne * sizeof(double));
    free(vc); free(cv); free(tv); free(vdeg); free(vptr); free(vedge);
}

/* The 3D toric code's face Tanner graph in CSR form: check f owns Tanner
 * edges 4f..4f+3, which join it to t3o_face_edges(f) in that order. */
void t3o_toric_tanner(int L, int32_t* cptr, int32_t* cvar)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t f = 0; f <= n; ++f) cptr[f] = (int32_t)(4 * f);
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        t3o_face_edges(L, f, ed);
        for (int j = 0; j < 4; ++j) cvar[4 * f + j] = (int32_t)ed[j];
    }
}

static double prior_llr(double p) { return log((1.0 - p) / p); }

/* BP on the toric code for one sample, then the hard decision of Sec. 4.1
 * (correct every qubit with l_v < 0): e ^= d, s ^= H d.  Returns nothing;
 * llr (optional, 3L^3) receives the posteriors. */
void t3o_bp_decode(int L, uint8_t* e, uint8_t* s, double p, double q, int meas_nodes,
                   int iters, double* llr_out)
{
    int64_t n = 3LL * L * L * L;
    int32_t* cptr = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* cvar = (int32_t*)malloc((size_t)(4 * n) * sizeof(int32_t));
    double* llr = (double*)malloc((size_t)n * sizeof(double));
    t3o_toric_tanner(L, cptr, cvar);
    double lq = (meas_nodes && q > 0.0) ? prior_llr(q) : INFINITY;
    t3o_bp((int)n, (int)n, cptr, cvar, s, prior_llr(p), lq, iters, NULL, NULL, llr);
    for (int64_t v = 0; v < n; ++v) {
        if (llr_out) llr_out[v] = llr[v];
        if (llr[v] < 0.0) {
            e[v] ^= 1;
        }
    }
    /* s ^= H d, face by face */
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        t3o_face_edges(L, f, ed);
        int par = 0;
        for (int j = 0; j < 4; ++j) par ^= (llr[ed[j]] < 0.0);
        s[f] ^= (uint8_t)par;
    }
    free(cptr); free(cvar); free(llr);
}

/* ------------------------------------------------------------------ */
/* BP on a factor graph with one prior LLR per variable (Sec. 4.1, Eqs. */
/* 1-4), the same flooding schedule and numerical guards as t3o_bp but  */
/* with every variable explicit: used for BP with meta-checks, where    */
/* the measurement-error variables have degree 3 instead of 1.          */
/* ------------------------------------------------------------------ */
void t3o_bp_priors_from(int nv, int nc, const int32_t* cptr, const int32_t* cvar, const uint8_t* syn,
                        const double* prior, int iters, const double* cv_in, double* cv_out, double* llr);

void t3o_bp_priors(int nv, int nc, const int32_t* cptr, const int32_t* cvar, const uint8_t* syn,
                   const double* prior, int iters, double* llr)
{
    t3o_bp_priors_from(nv, nc, cptr, cvar, syn, prior, iters, NULL, NULL, llr);
}

/* The same iterations started from given check->variable messages cv_in (one
 * per Tanner edge t = cptr[c] + k; NULL: all zero, the start above), leaving
 * the last ones in cv_out (nullable). */
void t3o_bp_priors_from(int nv, int nc, const int32_t* cptr, const int32_t* cvar, const uint8_t* syn,
                        const double* prior, int iters, const double* cv_in, double* cv_out, double* llr)
{
    int ne = cptr[nc];
    double* vc = (double*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
    double* cv = (double*)calloc((size_t)(ne > 0 ? ne : 1), sizeof(double));
    double* tv = (double*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
    int* vdeg = (int*)calloc((size_t)nv + 1, sizeof(int));
    int* vptr = (int*)calloc((size_t)nv + 1, sizeof(int));
    int* vedge = (int*)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(int));
    const double cap = 1.0 - 1e-15;

    if (cv_in) memcpy(cv, cv_in, (size_t)ne * sizeof(double));
    for (int t = 0; t < ne; ++t) vdeg[cvar[t]]++;
    for (int v = 0; v < nv; ++v) vptr[v + 1] = vptr[v] + vdeg[v];
    memset(vdeg, 0, (size_t)nv * sizeof(int));
    for (int t = 0; t < ne; ++t) {
        int v = cvar[t];
        vedge[vptr[v] + vdeg[v]++] = t;
    }
    for (int it = 0; it < iters; ++it) {
        /* variable -> check (Eq. 3; the prior alone on the first pass, when cv = 0) */
        for (int v = 0; v < nv; ++v)
            for (int i = vptr[v]; i < vptr[v + 1]; ++i) {
                double m = prior[v];
                for (int i2 = vptr[v]; i2 < vptr[v + 1]; ++i2)
                    if (i2 != i) m += cv[vedge[i2]];
                vc[vedge[i]] = m;
            }
        /* check -> variable (Eq. 2) */
        for (int t = 0; t < ne; ++t) tv[t] = tanh(vc[t] / 2.0);
        for (int c = 0; c < nc; ++c)
            for (int t = cptr[c]; t < cptr[c + 1]; ++t) {
                double prod = 1.0;
                for (int t2 = cptr[c]; t2 < cptr[c + 1]; ++t2)
                    if (t2 != t) prod *= tv[t2];
                if (prod > cap) prod = cap;
                if (prod < -cap) prod = -cap;
                double m = 2.0 * atanh(prod);
                if (syn[c] & 1) m = -m;
                if (m > 30.0) m = 30.0;
                if (m < -30.0) m = -30.0;
                cv[t] = m;
            }
    }
    /* posterior (Eq. 4) */
    if (llr)
        for (int v = 0; v < nv; ++v) {
            double l = prior[v];
            for (int i = vptr[v]; i < vptr[v + 1]; ++i) l += cv[vedge[i]];
            llr[v] = l;
        }
    if (cv_out) memcpy(cv_out, cv, (size_t)ne * sizeof(double));
    free(vc); free(cv); free(tv); free(vdeg); free(vptr); free(vedge);
}

/* The six faces of the unit cube at site r (spanning r .. r + e_x + e_y +
 * e_z): for each axis a the face with normal a at r and the one at
 * r + e_a.  Every face bounds exactly two cubes. */
void t3o_cube_faces(int L, int64_t site, int64_t out[6])
{
    int r[3] = { (int)(site % L), (int)((site / L) % L), (int)(site / ((int64_t)L * L)) };
    int64_t L3 = (int64_t)L * L * L;
    for (int a = 0; a < 3; ++a) {
        int q[3] = { r[0], r[1], r[2] };
        q[a] = (r[a] + 1) % L;
        out[2 * a] = a * L3 + site;
        out[2 * a + 1] = a * L3 + ((int64_t)q[2] * L + q[1]) * L + q[0];
    }
}

/* Meta-syndrome (Sec. 4.1, last paragraph): every error-free syndrome is a
 * union of closed loops, so the six faces of a cube have even parity; the
 * measured parity of cube c is the parity of the measurement errors on its
 * faces.  m: L^3 bytes. */
void t3o_meta_syndrome(int L, const uint8_t* s, uint8_t* m)
{
    int64_t L3 = (int64_t)L * L * L;
    for (int64_t c = 0; c < L3; ++c) {
        int64_t fc[6];
        t3o_cube_faces(L, c, fc);
        int par = 0;
        for (int j = 0; j < 6; ++j) par ^= s[fc[j]] & 1;
        m[c] = (uint8_t)par;
    }
}

/* Factor graph of BP with meta-checks in CSR form.  Variables 0..n-1 are
 * the qubits (edges), n + f the measurement error of face f.  Checks
 * 0..n-1 are the faces (their four edges in t3o_face_edges order, then
 * their measurement variable); checks n + c are the meta-checks, one per
 * cube, over the measurement variables of its six faces. */
void t3o_meta_tanner(int L, int32_t* cptr, int32_t* cvar)
{
    int64_t n = 3LL * L * L * L, L3 = (int64_t)L * L * L;
    int64_t t = 0;
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        cptr[f] = (int32_t)t;
        t3o_face_edges(L, f, ed);
        for (int j = 0; j < 4; ++j) cvar[t++] = (int32_t)ed[j];
        cvar[t++] = (int32_t)(n + f);
    }
    for (int64_t c = 0; c < L3; ++c) {
        int64_t fc[6];
        cptr[n + c] = (int32_t)t;
        t3o_cube_faces(L, c, fc);
        for (int j = 0; j < 6; ++j) cvar[t++] = (int32_t)(n + fc[j]);
    }
    cptr[n + L3] = (int32_t)t;
}

/* BP with meta-checks for one sample (qubit priors log((1-p)/p),
 * measurement priors log((1-q)/q)), then the hard decision on the qubits
 * as in t3o_bp_decode: e ^= d, s ^= H d.  llr_out (optional, 2 * 3L^3):
 * posteriors of the qubits, then of the measurement variables. */
void t3o_bp_meta_decode(int L, uint8_t* e, uint8_t* s, double p, double q, int iters, double* llr_out)
{
    int64_t n = 3LL * L * L * L, L3 = (int64_t)L * L * L;
    int64_t nc = n + L3, ne = 5 * n + 6 * L3;
    int32_t* cptr = (int32_t*)malloc((size_t)(nc + 1) * sizeof(int32_t));
    int32_t* cvar = (int32_t*)malloc((size_t)ne * sizeof(int32_t));
    uint8_t* syn = (uint8_t*)malloc((size_t)nc);
    double* prior = (double*)malloc((size_t)(2 * n) * sizeof(double));
    double* llr = (double*)malloc((size_t)(2 * n) * sizeof(double));
    t3o_meta_tanner(L, cptr, cvar);
    memcpy(syn, s, (size_t)n);
    t3o_meta_syndrome(L, s, syn + n);
    for (int64_t v = 0; v < n; ++v) {
        prior[v] = prior_llr(p);
        prior[n + v] = prior_llr(q);
    }
    t3o_bp_priors((int)(2 * n), (int)nc, cptr, cvar, syn, prior, iters, llr);
    for (int64_t v = 0; v < n; ++v)
        if (llr[v] < 0.0) e[v] ^= 1;
    for (int64_t f = 0; f < n; ++f) {
        int64_t ed[4];
        t3o_face_edges(L, f, ed);
        int par = 0;
        for (int j = 0; j < 4; ++j) par ^= (llr[ed[j]] < 0.0);
        s[f] ^= (uint8_t)par;
    }
    if (llr_out) memcpy(llr_out, llr, (size_t)(2 * n) * sizeof(double));
    free(cptr); free(cvar); free(syn); free(prior); free(llr);
}

void t3o_bp_meta_decode_batch(int L, int64_t n_samples, uint8_t* e, uint8_t* s, double p, double q,
                              int iters, double* llr)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_bp_meta_decode(L, e + i * n, s + i * n, p, q, iters, llr ? llr + i * 2 * n : NULL);
}

/* ------------------------------------------------------------------ */
/* Logical readout (Fig. 2 caption, Sec. 3.1 and its footnote, App. A.2):*/
/* for axis d the L^2 straight lines of d-edges (one per value of the   */
/* two other coordinates) are a complete disjoint set of logical Z      */
/* operators; each line reports the parity of the residual X error on   */
/* it and a majority of odd lines is a logical X error on qubit d.  A   */
/* tie (2c = L^2) counts as a failure.  Bit d of the result = axis d.   */
/* ------------------------------------------------------------------ */
int t3o_logical(int L, const uint8_t* e, int32_t* odd_counts)
{
    int mask = 0;
    for (int d = 0; d < 3; ++d) {
        int u = (d == 0) ? 1 : 0;   /* the two coordinates fixed along a line */
        int w = (d == 2) ? 1 : 2;
        int count = 0;
        for (int cu = 0; cu < L; ++cu) {
            for (int cw = 0; cw < L; ++cw) {
                int par = 0;
                for (int t = 0; t < L; ++t) {
                    int r[3];
                    r[d] = t; r[u] = cu; r[w] = cw;
                    par ^= e[edge_id(L, d, r)];
                }
                count += par & 1;
            }
        }
        if (odd_counts) odd_counts[d] = count;
        if (2 * count >= L * L) mask |= 1 << d;
    }
    return mask;
}

/* ------------------------------------------------------------------ */
/* A whole Monte Carlo run of one sample (Sec. 3.1 Fig. 2, Sec. 3.2     */
/* schedule list, Sec. 4.2 p-BP).  e starts at 0 (the paper does not    */
/* say; a fresh code).  For cycles t = cycle0+1 .. cycle0+T: qubit     */
/* noise, one noisy measurement, optional BP with hard decision, then  */
/* n_apply rule applications whose kinds cycle through the F/P        */
/* schedule string (Sec. 3.2 schedule list, Table 1 footnote, Sec. 4.2);*/
/* application k (counted from 0 within the cycle) keys the p-flip     */
/* coins.  Optionally a final noiseless measurement (cycle0+T+1) is     */
/* decoded by F applications until the syndrome is clear or            */
/* perfect_max_sweeps.  Returns the 3-bit logical mask.                */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t L;
    int32_t T;
    double p;
    double q;
    uint64_t seed;
    int32_t use_bp;
    int32_t bp_iters;
    int32_t bp_meas_nodes;
    int32_t n_apply;
    char schedule[64];
    int32_t perfect_round;
    int32_t perfect_max_sweeps;
    uint32_t cycle0;
    int32_t bp_meta;     /* 1: BP with meta-checks (needs q > 0) in place of plain BP */
} t3o_cfg;

static int syndrome_clear(int64_t n, const uint8_t* s)
{
    for (int64_t f = 0; f < n; ++f)
        if (s[f]) return 0;
    return 1;
}

/* e (3L^3 bytes) is both the initial state and the result. */
int t3o_run_sample(const t3o_cfg* cfg, uint64_t sample, uint8_t* e)
{
    const int L = cfg->L;
    const int64_t n = 3LL * L * L * L;
    uint8_t* s = (uint8_t*)calloc((size_t)n, 1);
    size_t slen = strnlen(cfg->schedule, sizeof(cfg->schedule));
    for (int t = 1; t <= cfg->T; ++t) {
        uint32_t cycle = cfg->cycle0 + (uint32_t)t;
        t3o_noise(L, e, cfg->p, cfg->seed, sample, cycle);
        t3o_measure(L, e, s, cfg->q, cfg->seed, sample, cycle);
        if (cfg->use_bp && cfg->bp_meta)
            t3o_bp_meta_decode(L, e, s, cfg->p, cfg->q, cfg->bp_iters, NULL);
        else if (cfg->use_bp)
            t3o_bp_decode(L, e, s, cfg->p, cfg->q, cfg->bp_meas_nodes, cfg->bp_iters, NULL);
        for (int k = 0; slen > 0 && k < cfg->n_apply; ++k) {
            if (cfg->schedule[(size_t)k % slen] == 'P')
                t3o_pflip_once(L, e, s, cfg->seed, sample, cycle, (uint32_t)k);
            else
                t3o_flip_once(L, e, s);
        }
    }
    if (cfg->perfect_round) {
        t3o_syndrome(L, e, s);
        for (int k = 0; k < cfg->perfect_max_sweeps && !syndrome_clear(n, s); ++k)
            t3o_flip_once(L, e, s);
    }
    free(s);
    return t3o_logical(L, e, NULL);
}

/* ------------------------------------------------------------------ */
/* Batch wrappers: loop the per-sample functions over samples stored   */
/* [sample][3L^3] (uint8) so the Python side makes one call per batch. */
/* ------------------------------------------------------------------ */
void t3o_run_batch(const t3o_cfg* cfg, uint64_t sample0, int64_t n_samples, uint8_t* e,
                   uint8_t* mask)
{
    int64_t n = 3LL * cfg->L * cfg->L * cfg->L;
    for (int64_t i = 0; i < n_samples; ++i)
        mask[i] = (uint8_t)t3o_run_sample(cfg, sample0 + (uint64_t)i, e + i * n);
}

void t3o_noise_batch(int L, int64_t n_samples, uint8_t* e, double p, uint64_t seed,
                     uint64_t sample0, uint32_t cycle)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_noise(L, e + i * n, p, seed, sample0 + (uint64_t)i, cycle);
}

void t3o_measure_batch(int L, int64_t n_samples, const uint8_t* e, uint8_t* s, double q,
                       uint64_t seed, uint64_t sample0, uint32_t cycle)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_measure(L, e + i * n, s + i * n, q, seed, sample0 + (uint64_t)i, cycle);
}

void t3o_syndrome_batch(int L, int64_t n_samples, const uint8_t* e, uint8_t* s)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i) t3o_syndrome(L, e + i * n, s + i * n);
}

void t3o_flip_batch(int L, int64_t n_samples, uint8_t* e, uint8_t* s, int probabilistic,
                    uint64_t seed, uint64_t sample0, uint32_t cycle, uint32_t sweep)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i)
        apply_rule(L, e + i * n, s + i * n, probabilistic, seed, sample0 + (uint64_t)i,
                   cycle, sweep);
}

void t3o_logical_batch(int L, int64_t n_samples, const uint8_t* e, uint8_t* mask)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i) mask[i] = (uint8_t)t3o_logical(L, e + i * n, NULL);
}

/* BP on a batch: s (n_samples x 3L^3 bytes) in, messages and posteriors out,
 * messages [sample][4*3L^3] in Tanner-edge order of t3o_toric_tanner. */
void t3o_bp_batch(int L, int64_t n_samples, const uint8_t* s, double p, double q,
                  int meas_nodes, int iters, const double* m_in, double* m_out, double* llr)
{
    int64_t n = 3LL * L * L * L;
    int32_t* cptr = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* cvar = (int32_t*)malloc((size_t)(4 * n) * sizeof(int32_t));
    t3o_toric_tanner(L, cptr, cvar);
    double lq = (meas_nodes && q > 0.0) ? prior_llr(q) : INFINITY;
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_bp((int)n, (int)n, cptr, cvar, s + i * n, prior_llr(p), lq, iters,
               m_in ? m_in + i * 4 * n : NULL, m_out ? m_out + i * 4 * n : NULL,
               llr ? llr + i * n : NULL);
    free(cptr); free(cvar);
}

void t3o_bp_decode_batch(int L, int64_t n_samples, uint8_t* e, uint8_t* s, double p, double q,
                         int meas_nodes, int iters, double* llr)
{
    int64_t n = 3LL * L * L * L;
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_bp_decode(L, e + i * n, s + i * n, p, q, meas_nodes, iters, llr ? llr + i * n : NULL);
}

int t3o_abi_version(void) { return 1; }

/* ------------------------------------------------------------------ */
/* Generic Tanner graphs (Sec. 5 asks whether these decoders carry over */
/* to other LDPC codes).  A code is given by its checks in CSR form:    */
/* check c acts on variables cvar[cptr[c]] .. cvar[cptr[c+1]-1].  The   */
/* rules are the toric code's, stated per variable: flip a variable     */
/* when more of its checks are unsatisfied than satisfied (Sec. 3.1);   */
/* p-flip also flips, with probability 1/2, a variable with exactly as  */
/* many unsatisfied as satisfied checks (Sec. 3.2).  Noise keys the     */
/* generator with the variable index as site (stream 0), measurement    */
/* errors with the check index (stream 1), as on the toric code.  The   */
/* p-flip coin of variable v is bit `lane` of word v mod 4 of stream 2 */
/* keyed by site v / 4 (two blocks serve four variables).               */
/* ------------------------------------------------------------------ */
void t3o_tanner_syndrome(int64_t m, const int32_t* cptr, const int32_t* cvar, const uint8_t* e, uint8_t* s)
{
    for (int64_t c = 0; c < m; ++c) {
        uint8_t par = 0;
        for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) par ^= e[cvar[t]];
        s[c] = par;
    }
}

void t3o_tanner_noise(int64_t n, uint8_t* e, double p, uint64_t seed, uint64_t sample, uint32_t cycle)
{
    for (int64_t v = 0; v < n; ++v)
        if (t3o_bernoulli(p, seed, STREAM_QUBIT, (uint64_t)v, cycle, 0, sample)) e[v] ^= 1;
}

void t3o_tanner_measure(int64_t m, const int32_t* cptr, const int32_t* cvar, const uint8_t* e, uint8_t* s,
                        double q, uint64_t seed, uint64_t sample, uint32_t cycle)
{
    t3o_tanner_syndrome(m, cptr, cvar, e, s);
    for (int64_t c = 0; c < m; ++c)
        if (t3o_bernoulli(q, seed, STREAM_MEAS, (uint64_t)c, cycle, 0, sample)) s[c] ^= 1;
}

int t3o_tanner_coin(uint64_t seed, int64_t v, uint32_t cycle, uint32_t sweep, uint64_t sample)
{
    return t3o_coin(seed, (uint64_t)(v / 4), (int)(v % 4), cycle, sweep, sample);
}

/* One parallel application: every variable decides from the same syndrome, then e ^= f, s ^= H f. */
void t3o_tanner_rule(int64_t n, int64_t m, const int32_t* cptr, const int32_t* cvar, uint8_t* e, uint8_t* s,
                     int probabilistic, uint64_t seed, uint64_t sample, uint32_t cycle, uint32_t sweep)
{
    int32_t* deg = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int32_t* unsat = (int32_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    uint8_t* flip = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t c = 0; c < m; ++c)
        for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) {
            deg[cvar[t]]++;
            unsat[cvar[t]] += s[c];
        }
    for (int64_t v = 0; v < n; ++v) {
        int sat = deg[v] - unsat[v];
        if (unsat[v] > sat)
            flip[v] = 1;
        else if (probabilistic && unsat[v] == sat && deg[v] > 0)
            flip[v] = (uint8_t)t3o_tanner_coin(seed, v, cycle, sweep, sample);
    }
    for (int64_t v = 0; v < n; ++v) e[v] ^= flip[v];
    for (int64_t c = 0; c < m; ++c)
        for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) s[c] ^= flip[cvar[t]];
    free(deg); free(unsat); free(flip);
}

void t3o_tanner_syndrome_batch(int64_t n, int64_t m, const int32_t* cptr, const int32_t* cvar, int64_t n_samples,
                               const uint8_t* e, uint8_t* s)
{
    for (int64_t i = 0; i < n_samples; ++i) t3o_tanner_syndrome(m, cptr, cvar, e + i * n, s + i * m);
}

void t3o_tanner_noise_batch(int64_t n, int64_t n_samples, uint8_t* e, double p, uint64_t seed, uint64_t sample0,
                            uint32_t cycle)
{
    for (int64_t i = 0; i < n_samples; ++i) t3o_tanner_noise(n, e + i * n, p, seed, sample0 + (uint64_t)i, cycle);
}

void t3o_tanner_measure_batch(int64_t n, int64_t m, const int32_t* cptr, const int32_t* cvar, int64_t n_samples,
                              const uint8_t* e, uint8_t* s, double q, uint64_t seed, uint64_t sample0,
                              uint32_t cycle)
{
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_tanner_measure(m, cptr, cvar, e + i * n, s + i * m, q, seed, sample0 + (uint64_t)i, cycle);
}

void t3o_tanner_rule_batch(int64_t n, int64_t m, const int32_t* cptr, const int32_t* cvar, int64_t n_samples,
                           uint8_t* e, uint8_t* s, int probabilistic, uint64_t seed, uint64_t sample0,
                           uint32_t cycle, uint32_t sweep)
{
    for (int64_t i = 0; i < n_samples; ++i)
        t3o_tanner_rule(n, m, cptr, cvar, e + i * n, s + i * m, probabilistic, seed, sample0 + (uint64_t)i,
                        cycle, sweep);
}

/* BP with one prior per variable on a batch: syndromes s (n_samples x m), posteriors
 * llr (n_samples x n), hard decision applied: e ^= d, s ^= H d. */
void t3o_tanner_bp_batch(int64_t n, int64_t m, const int32_t* cptr, const int32_t* cvar, int64_t n_samples,
                         uint8_t* e, uint8_t* s, const double* prior, int iters, double* llr)
{
    double* l = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    uint8_t* d = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n_samples; ++i) {
        t3o_bp_priors((int)n, (int)m, cptr, cvar, s + i * m, prior, iters, l);
        for (int64_t v = 0; v < n; ++v) {
            d[v] = l[v] < 0.0;
            e[i * n + v] ^= d[v];
        }
        for (int64_t c = 0; c < m; ++c)
            for (int32_t t = cptr[c]; t < cptr[c + 1]; ++t) s[i * m + c] ^= d[cvar[t]];
        if (llr) memcpy(llr + i * n, l, (size_t)n * sizeof(double));
    }
    free(l); free(d);
}
