// fd_weights.cpp -- the FD-coefficient generator of libwave.so.
//
// Centred second-derivative weights of accuracy order SO on unit spacing
// (the coefficients printed in McCormick 2017, Fig. acoustic_devito, for
// SO = 8, there multiplied by 2dt^2/h^2):
//     a_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!),  k = 1..r,  r = SO/2,
//     a_0 = -2 sum_k a_k.
// Computed as exact fractions (128-bit numerators and denominators, reduced
// by gcd), then rounded once to double.
#include <cmath>
#include <cstdlib>

#include "wave_host.h"

namespace wave {
namespace {

using i128 = __int128;

i128 gcd128(i128 a, i128 b)
{
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
        i128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

struct Frac {
    i128 num, den;  // den > 0, reduced
};

Frac make(i128 n, i128 d)
{
    if (d < 0) { n = -n; d = -d; }
    i128 g = gcd128(n, d);
    if (g > 1) { n /= g; d /= g; }
    return {n, d};
}

Frac add(Frac a, Frac b)
{
    i128 g = gcd128(a.den, b.den);
    i128 l = a.den / g * b.den;
    return make(a.num * (l / a.den) + b.num * (l / b.den), l);
}

double to_double(Frac f)
{
    // numerators and denominators stay far below 2^63 for r <= 8
    return static_cast<double>(static_cast<long long>(f.num)) / static_cast<double>(static_cast<long long>(f.den));
}

bool weights_frac(int so, Frac* a)
{
    if (so < 2 || so > 16 || (so & 1)) return false;
    const int r = so / 2;
    Frac sum = {0, 1};
    for (int k = 1; k <= r; ++k) {
        // (r!)^2 / ((r-k)! (r+k)!) = prod_{i<k} (r - i) / prod_{i=1..k} (r + i)
        i128 num = 2, den = static_cast<i128>(k) * k;
        for (int i = 0; i < k; ++i) num *= (r - i);
        for (int i = 1; i <= k; ++i) den *= (r + i);
        if ((k + 1) % 2) num = -num;
        a[k] = make(num, den);
        sum = add(sum, a[k]);
    }
    a[0] = make(-2 * sum.num, sum.den);
    return true;
}

}  // namespace

bool fd_weights_exact(int so, double* out)
{
    Frac a[9];
    if (!weights_frac(so, a)) return false;
    for (int k = 0; k <= so / 2; ++k) out[k] = to_double(a[k]);
    return true;
}

double fd_spectral_radius(int so)
{
    Frac a[9];
    if (!weights_frac(so, a)) return 0.0;
    Frac rho = make(a[0].num < 0 ? -a[0].num : a[0].num, a[0].den);
    for (int k = 1; k <= so / 2; ++k) {
        Frac t = make(2 * (a[k].num < 0 ? -a[k].num : a[k].num), a[k].den);
        rho = add(rho, t);
    }
    return to_double(rho);
}

}  // namespace wave

extern "C" wave_status wave_fd_weights(int so, double* a)
{
    if (!a) return wave::fail(WAVE_ERR_ARG, "wave_fd_weights: null output");
    if (!wave::fd_weights_exact(so, a)) return wave::fail(WAVE_ERR_ARG, "wave_fd_weights: so must be even, 2..16");
    return WAVE_OK;
}

extern "C" wave_status wave_cfl_limit(int so, const double spacing[3], double vmax, double* dt_max)
{
    if (!spacing || !dt_max) return wave::fail(WAVE_ERR_ARG, "wave_cfl_limit: null argument");
    if (!(vmax > 0.0) || !(spacing[0] > 0.0) || !(spacing[1] > 0.0) || !(spacing[2] > 0.0))
        return wave::fail(WAVE_ERR_ARG, "wave_cfl_limit: vmax and spacing must be positive");
    const double rho = wave::fd_spectral_radius(so);
    if (rho <= 0.0) return wave::fail(WAVE_ERR_ARG, "wave_cfl_limit: so must be even, 2..16");
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += rho / (spacing[a] * spacing[a]);
    // leapfrog on u_tt = v^2 L u is stable iff dt^2 v^2 lambda_max <= 4
    *dt_max = 2.0 / (vmax * std::sqrt(s));
    return WAVE_OK;
}
