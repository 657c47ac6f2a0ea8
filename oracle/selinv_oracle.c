/*
 * CPU oracle for supernodal selected inversion (Jacquelin, Lin, Jia, Zhao,
 * Yang, "A left-looking selected inversion algorithm and task parallelism on
 * shared memory systems").
 *
 * TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It is plain C with
 * no BLAS, written from the paper's definitions and algorithms, and shares
 * no code with the GPU library.  Real values are double, complex values are
 * double _Complex (complex symmetric: plain transposes; the _h entry points
 * take complex Hermitian matrices: conjugate transposes).
 *
 * Entry points (suffix _d: real, _z: complex symmetric, _h: complex Hermitian --
 * orc_ldlt_h and orc_selinv_h / orc_selinv_top_h only):
 *   orc_symbolic / orc_sym_get / orc_sym_free / orc_plan  (oracle_symbolic.c)
 *   orc_ldlt_*          supernodal-pattern LDL^T, no pivoting (Sec. IV prerequisite)
 *   orc_selinv_*        Alg. 1 (pull), symmetrized diagonal blocks (Sec. II-C)
 *   orc_selinv_levels_* the same steps, the supernodes of one tree level on
 *                       host threads at a time (bit for bit orc_selinv)
 *   orc_selinv_push_*   Alg. 2 (left-looking push: outer/inner products)
 *   orc_selinv_adjoint_*, orc_ldlt_adjoint_*   reverse mode of the two above
 */
#include <complex.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)

#define T double
#define SFX _d
#define CJ(x) (x)
#define HERM 0
#include "oracle_numeric.inc"
#undef T
#undef SFX
#undef CJ
#undef HERM

#define T double _Complex
#define SFX _z
#define CJ(x) (x)
#define HERM 0
#include "oracle_numeric.inc"
#undef T
#undef SFX
#undef CJ
#undef HERM

#define T double _Complex
#define SFX _h
#define CJ(x) conj(x)
#define HERM 1
#include "oracle_numeric.inc"
#undef T
#undef SFX
#undef CJ
#undef HERM

int orc_version(void) { return 1; }
