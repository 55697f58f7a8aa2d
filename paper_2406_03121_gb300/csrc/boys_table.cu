// Host-side tabulation of the Boys function grid used by the kernels:
//   tab[k][n] = F_n(T_k), T_k = k * MESS_BOYS_DT, n = 0..MESS_BOYS_NF-1;  tab[k][MESS_BOYS_NF] = exp(-T_k).
// F_{NF-1}(T) comes from the positive series exp(-T) sum_i (2T)^i / ((2n+1)(2n+3)...(2n+2i+1)) in
// long double; the lower orders follow from the downward recursion F_{n-1} = (2T F_n + e^{-T})/(2n-1),
// which is stable in that direction.
#include <math.h>

#include <vector>

#include "mess_internal.h"

void mess_boys_table(std::vector<double>& tab, int nrow, double dt)
{
    tab.assign((size_t)nrow * MESS_BOYS_NCOL, 0.0);
    for (int k = 0; k < nrow; ++k) {
        const long double T = (long double)k * (long double)dt;
        const long double eT = expl(-T);
        const int top = MESS_BOYS_NF - 1;
        long double term = 1.0L / (2 * top + 1), sum = term;
        for (int i = 1; i < 10000; ++i) {
            term *= 2.0L * T / (long double)(2 * top + 2 * i + 1);
            sum += term;
            if (term < sum * 1e-21L) break;
        }
        long double F[MESS_BOYS_NF];
        F[top] = eT * sum;
        for (int n = top; n >= 1; --n) F[n - 1] = (2.0L * T * F[n] + eT) / (long double)(2 * n - 1);
        for (int n = 0; n < MESS_BOYS_NF; ++n) tab[(size_t)k * MESS_BOYS_NCOL + n] = (double)F[n];
        tab[(size_t)k * MESS_BOYS_NCOL + MESS_BOYS_NF] = (double)eT;
    }
}

extern "C" mess_status mess_boys_grid(double* out, int max_values, int* nrows, int* ncols, double* dT)
{
    if (nrows) *nrows = MESS_BOYS_NROW;
    if (ncols) *ncols = MESS_BOYS_NCOL;
    if (dT) *dT = MESS_BOYS_DT;
    if (!out) return MESS_OK;
    if (max_values < MESS_BOYS_NROW * MESS_BOYS_NCOL) {
        mess_set_error("mess_boys_grid: %d values needed, max_values = %d", MESS_BOYS_NROW * MESS_BOYS_NCOL, max_values);
        return MESS_EINVAL;
    }
    std::vector<double> tab;
    mess_boys_table(tab, MESS_BOYS_NROW, MESS_BOYS_DT);
    for (size_t i = 0; i < tab.size(); ++i) out[i] = tab[i];
    return MESS_OK;
}
