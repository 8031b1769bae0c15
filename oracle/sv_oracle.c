/*
 * FP64 CPU oracle for the state-vector gate update.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the bench's CPU-baseline leg call it; the library never does.  It shares no code with the CUDA path.
 *
 * What it computes (paper, Sec. V.A): the state is the vector of 2^n amplitudes alpha_k, qubit t is bit t
 * of the index k (stride 2^t, Fig. "statevector" caption).  A single-qubit gate Q = [[q11, q12], [q21, q22]]
 * on qubit t replaces every pair (alpha_k, alpha_{k+2^t}) with k's bit t equal to 0 by
 *     alpha_k        <- q11 alpha_k + q12 alpha_{k+2^t}
 *     alpha_{k+2^t}  <- q21 alpha_k + q22 alpha_{k+2^t}
 * (the strided pair-update equation), both right-hand sides taken from the old values.  The pairs are
 * visited in the order of Algorithm 1: an outer loop over blocks of 2^(t+1) amplitudes and an inner loop
 * over the first 2^t amplitudes of each block.  A controlled gate does the same update only at indices
 * whose control bits are all 1 (Sec. V.B, the caption of the gate-application algorithm).
 *
 * SWAP of qubits a and b exchanges alpha_k and alpha_{k xor 2^a xor 2^b} wherever bit a of k is 1 and bit b
 * is 0; Sec. VI.B's "non-sequential storage" example (n = 3, order 0,1,4,5,2,3,6,7) is SWAP(1, 2).
 *
 * A two-qubit gate (Sec. II.B: multi-qubit gates such as CNOT act as 4x4 matrices on the four basis states
 * of their qubits) is a 4x4 matrix V on qubits q0 and q1: for every index k whose bits q0 and q1 are 0 (and
 * whose control bits are all 1), the four amplitudes alpha_{k + b0 2^q0 + b1 2^q1} form a vector a indexed by
 * j = b0 + 2 b1, replaced by V a (old values on the right, the sum over j taken in order 0..3).
 *
 * Plain C99, IEEE double, no fused multiply-add (built with -ffp-contract=off), no reordering beyond the
 * loop order above.  The amplitudes are stored interleaved (re, im) in a double array of length 2^(n+1).
 *
 * Threads: the timing entry point may split the outer loop over OpenMP threads (the paper's "outer"
 * variant, Sec. V.B.2); every pair is independent, so the result does not depend on the thread count.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)

#define KIND_U 0
#define KIND_SWAP 1
#define KIND_U4 2
#define KIND_U4_ROW 3

/* Byte layout of one gate record: 96 bytes, the same as the input generator's record. */
typedef struct {
    double U[8]; /* q11, q12, q21, q22 as (re, im) */
    int32_t kind;
    int32_t target;
    int32_t target2;
    int32_t ncontrols;
    int32_t controls[4];
} oracle_gate;

int oracle_gate_size(void) { return (int)sizeof(oracle_gate); }

/* |x>: every amplitude 0 except alpha_x = 1 (computational basis, Sec. II.A). */
int oracle_init_basis(int n, double *psi, uint64_t x)
{
    if (n < 1 || n > 40 || psi == NULL) return ORACLE_ERR_ARG;
    uint64_t dim = (uint64_t)1 << n;
    if (x >= dim) return ORACLE_ERR_ARG;
    memset(psi, 0, sizeof(double) * 2 * dim);
    psi[2 * x] = 1.0;
    return ORACLE_OK;
}

/* The pair update of Sec. V.A on a = alpha_k and b = alpha_{k+2^t}, both outputs from the old values:
 * alpha_k <- q11 a + q12 b ; alpha_{k+2^t} <- q21 a + q22 b  (complex products written out). */
static void pair_update(double *a, double *b, const double *U)
{
    const double q11r = U[0], q11i = U[1], q12r = U[2], q12i = U[3];
    const double q21r = U[4], q21i = U[5], q22r = U[6], q22i = U[7];
    const double ar = a[0], ai = a[1], br = b[0], bi = b[1];
    a[0] = (q11r * ar - q11i * ai) + (q12r * br - q12i * bi);
    a[1] = (q11r * ai + q11i * ar) + (q12r * bi + q12i * br);
    b[0] = (q21r * ar - q21i * ai) + (q22r * br - q22i * bi);
    b[1] = (q21r * ai + q21i * ar) + (q22r * bi + q22i * br);
}

/* The controlled-gate rule of Sec. V.B: the update applies only where every control bit of k is 1. */
static int controls_on(uint64_t k, uint64_t cmask) { return (k & cmask) == cmask; }

/* One gate: Algorithm 1's double loop with the controlled-gate test on each visited index. */
static int apply_u(int n, double *psi, const double *U, int t, const int32_t *controls, int nc, int nthreads,
                   int collapse)
{
    if (t < 0 || t >= n || nc < 0 || nc > 4) return ORACLE_ERR_ARG;
    uint64_t cmask = 0;
    for (int i = 0; i < nc; ++i) {
        if (controls[i] < 0 || controls[i] >= n || controls[i] == t) return ORACLE_ERR_ARG;
        if (cmask & ((uint64_t)1 << controls[i])) return ORACLE_ERR_ARG;
        cmask |= (uint64_t)1 << controls[i];
    }
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t stride = (uint64_t)1 << t;           /* 2^t: distance between the two amplitudes of a pair */
    const uint64_t nblocks = dim / (2 * stride);         /* outer loop: j = 0, 2^(t+1), 2*2^(t+1), ... */
    (void)nthreads;
    int64_t jb, kk;
    if (collapse && nthreads > 1) {
        /* The paper's collapse(2) variant (Sec. V.B.2): both loops of Algorithm 1 shared by the threads, so a
         * gate on a high qubit (few outer blocks) is split as finely as one on qubit 0.  Every pair is updated
         * exactly as below; only the thread that does it differs. */
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads)
        for (jb = 0; jb < (int64_t)nblocks; ++jb) {
            for (kk = 0; kk < (int64_t)stride; ++kk) {
                const uint64_t k = (uint64_t)jb * 2 * stride + (uint64_t)kk;
                if (!controls_on(k, cmask)) continue;
                pair_update(psi + 2 * k, psi + 2 * (k + stride), U);
            }
        }
        return ORACLE_OK;
    }
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1) if (nthreads > 1)
    for (jb = 0; jb < (int64_t)nblocks; ++jb) {
        const uint64_t j = (uint64_t)jb * 2 * stride;
        for (uint64_t k = j; k < j + stride; ++k) {       /* inner loop: k pairs with k + 2^t */
            if (!controls_on(k, cmask)) continue;           /* controlled gate: all control bits must be 1 */
            pair_update(psi + 2 * k, psi + 2 * (k + stride), U);
        }
    }
    return ORACLE_OK;
}

/* SWAP(a, b): exchange the amplitudes of the two index sets that differ only by bits a and b. */
static int apply_swap(int n, double *psi, int qa, int qb)
{
    if (qa < 0 || qa >= n || qb < 0 || qb >= n || qa == qb) return ORACLE_ERR_ARG;
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t ma = (uint64_t)1 << qa, mb = (uint64_t)1 << qb;
    for (uint64_t k = 0; k < dim; ++k) {
        if ((k & ma) && !(k & mb)) {
            uint64_t k2 = k ^ ma ^ mb;
            double r = psi[2 * k], i = psi[2 * k + 1];
            psi[2 * k] = psi[2 * k2];
            psi[2 * k + 1] = psi[2 * k2 + 1];
            psi[2 * k2] = r;
            psi[2 * k2 + 1] = i;
        }
    }
    return ORACLE_OK;
}

/* Two-qubit gate: V holds 16 complex entries row-major as (re, im); entry (r, j) multiplies the amplitude whose
 * (b0, b1) spell j = b0 + 2 b1 into the output whose bits spell r. */
static int apply_u4(int n, double *psi, const double *V, int q0, int q1, const int32_t *controls, int nc)
{
    if (q0 < 0 || q0 >= n || q1 < 0 || q1 >= n || q0 == q1 || nc < 0 || nc > 4) return ORACLE_ERR_ARG;
    uint64_t cmask = 0;
    for (int i = 0; i < nc; ++i) {
        if (controls[i] < 0 || controls[i] >= n || controls[i] == q0 || controls[i] == q1) return ORACLE_ERR_ARG;
        if (cmask & ((uint64_t)1 << controls[i])) return ORACLE_ERR_ARG;
        cmask |= (uint64_t)1 << controls[i];
    }
    const uint64_t dim = (uint64_t)1 << n;
    const uint64_t m0 = (uint64_t)1 << q0, m1 = (uint64_t)1 << q1;
    for (uint64_t k = 0; k < dim; ++k) {
        if (k & (m0 | m1)) continue;                     /* k = the member of the quadruple with b0 = b1 = 0 */
        if (cmask != (k & cmask)) continue;              /* every control bit must be 1 */
        uint64_t idx[4];
        double ar[4], ai[4];
        for (int j = 0; j < 4; ++j) {
            idx[j] = k | ((j & 1) ? m0 : 0) | ((j & 2) ? m1 : 0);
            ar[j] = psi[2 * idx[j]];
            ai[j] = psi[2 * idx[j] + 1];
        }
        for (int r = 0; r < 4; ++r) {
            double sr = 0.0, si = 0.0;
            for (int j = 0; j < 4; ++j) {
                const double vr = V[8 * r + 2 * j], vi = V[8 * r + 2 * j + 1];
                sr = sr + (vr * ar[j] - vi * ai[j]);
                si = si + (vr * ai[j] + vi * ar[j]);
            }
            psi[2 * idx[r]] = sr;
            psi[2 * idx[r] + 1] = si;
        }
    }
    return ORACLE_OK;
}

int oracle_apply_gate4(int n, double *psi, const double *V, int q0, int q1, const int32_t *controls, int ncontrols)
{
    if (n < 1 || n > 40 || psi == NULL || V == NULL) return ORACLE_ERR_ARG;
    if (ncontrols > 0 && controls == NULL) return ORACLE_ERR_ARG;
    return apply_u4(n, psi, V, q0, q1, controls, ncontrols);
}

int oracle_apply_gate(int n, double *psi, const double *U, int target, const int32_t *controls, int ncontrols)
{
    if (n < 1 || n > 40 || psi == NULL || U == NULL) return ORACLE_ERR_ARG;
    if (ncontrols > 0 && controls == NULL) return ORACLE_ERR_ARG;
    return apply_u(n, psi, U, target, controls, ncontrols, 1, 0);
}

int oracle_apply_swap(int n, double *psi, int a, int b)
{
    if (n < 1 || n > 40 || psi == NULL) return ORACLE_ERR_ARG;
    return apply_swap(n, psi, a, b);
}

/* A circuit is its gates applied one after another (Sec. II.B).  Returns the index of the first bad gate
 * as -(index + 2) on error, ORACLE_OK otherwise. */
static int apply_circuit(int n, double *psi, const oracle_gate *g, uint64_t ngates, int nthreads, int collapse)
{
    if (n < 1 || n > 40 || psi == NULL || (ngates > 0 && g == NULL)) return ORACLE_ERR_ARG;
    for (uint64_t i = 0; i < ngates; ++i) {
        int rc;
        if (g[i].kind == KIND_SWAP) rc = apply_swap(n, psi, g[i].target, g[i].target2);
        else if (g[i].kind == KIND_U)
            rc = apply_u(n, psi, g[i].U, g[i].target, g[i].controls, g[i].ncontrols, nthreads, collapse);
        else if (g[i].kind == KIND_U4 && i + 3 < ngates) {
            /* the matrix's four rows come from this record and the next three */
            double V[32];
            rc = ORACLE_OK;
            for (int r = 0; r < 4; ++r) {
                if (r > 0 && g[i + r].kind != KIND_U4_ROW) rc = ORACLE_ERR_ARG;
                memcpy(V + 8 * r, g[i + r].U, sizeof(double) * 8);
            }
            if (rc == ORACLE_OK) rc = apply_u4(n, psi, V, g[i].target, g[i].target2, g[i].controls, g[i].ncontrols);
            if (rc == ORACLE_OK) i += 3;
        }
        else rc = ORACLE_ERR_ARG;
        if (rc != ORACLE_OK) return -(int)(i + 2);
    }
    return ORACLE_OK;
}

int oracle_apply_circuit(int n, double *psi, const oracle_gate *g, uint64_t ngates, int nthreads)
{
    return apply_circuit(n, psi, g, ngates, nthreads, 0);
}

/* The same with the one-qubit gates' two loops collapsed over the threads (Sec. V.B.2's collapse variant);
 * the result is bit-identical to the sequential one. */
int oracle_apply_circuit_collapse(int n, double *psi, const oracle_gate *g, uint64_t ngates, int nthreads)
{
    return apply_circuit(n, psi, g, ngates, nthreads, 1);
}

/* Sum of |alpha_k|^2 (the normalisation condition of Sec. II.A), accumulated in index order. */
double oracle_norm2(int n, const double *psi)
{
    const uint64_t dim = (uint64_t)1 << n;
    double s = 0.0;
    for (uint64_t k = 0; k < dim; ++k) s += psi[2 * k] * psi[2 * k] + psi[2 * k + 1] * psi[2 * k + 1];
    return s;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
