/* Test infrastructure (the oracle): log r and exp(-r) evaluated element by
 * element by the platform C library.
 *
 * The paper's kernels log r (§6.1.1) and exp(-r) (App. D) are elementary
 * functions whose last bit depends on the implementation.  The pivots of the
 * NCA / ACA construction are argmax decisions on kernel values; on point sets
 * with exact ties (tensor grids) the last bit decides them.  The oracle takes
 * these two functions from the C library so that it breaks every tie on the
 * same values as any C or C++ construction built on the same library. */
#include <math.h>

void oracle_log(const double* r, double* out, long n) {
    for (long i = 0; i < n; ++i) out[i] = log(r[i]);
}

void oracle_exp_neg(const double* r, double* out, long n) {
    for (long i = 0; i < n; ++i) out[i] = exp(-r[i]);
}
