// Host build of the library's multi-limb arithmetic (csrc/mp.cuh, compiled here with
// shims that map the device rounding intrinsics to the identical IEEE operations of the
// host) on adversarial operands: heavy cancellation in additions, products, running
// sums.  Prints operands and results as hex floats for an exact check in Python.
#include <cstdio>
#include <cstdlib>
#include <random>
#include "mp_host.h"
using namespace hc;
static std::mt19937_64 rng(20261204);
static double urand() { return std::uniform_real_distribution<double>(-1.0, 1.0)(rng); }
template <int L> static R<L> rand_r(double scale)
{
    R<L> r;
    r.v[0] = urand() * scale;
    for (int k = 1; k < L; k++) r.v[k] = r.v[k - 1] * 0x1p-53 * urand();
    return L == 4 ? (R<L>)renorm5_pass(r.v[0], r.v[1 % L], r.v[2 % L], r.v[3 % L], 0.0) : r;
}
template <> R<2> rand_r<2>(double scale)
{
    R<2> r;
    double a = urand() * scale, b = a * 0x1p-53 * urand();
    fast_two_sum(a, b, r.v[0], r.v[1]);
    return r;
}
template <int L> static void out(const R<L> &r) { for (int k = 0; k < L; k++) printf("%a ", r.v[k]); }
template <int L> static void run(int mode, int count)
{
    for (int i = 0; i < count; i++) {
        R<L> a = rand_r<L>(1.0), b, r;
        if (mode == 0) {          // a + b, b = -(a + d): cancellation down to d's order
            R<L> d = rand_r<L>(std::ldexp(1.0, -(int)(rng() % (L == 4 ? 200 : 100))));
            b = r_neg(r_add(a, d));
            r = r_add(a, b);
        } else if (mode == 1) {   // the top of the sum cancels exactly: leading limbs one unit apart
            const double u = std::ldexp(1.0, std::ilogb(a.v[0]) - 52);
            b.v[0] = -(a.v[0] + u);
            for (int k = 1; k < L; k++) b.v[k] = -a.v[k] * (1 + urand() * 0x1p-30);
            b.v[1] += u;
            r = r_add(a, b);
        } else if (mode == 2) {   // a * b
            b = rand_r<L>(std::ldexp(1.0, (int)(rng() % 40) - 20));
            r = r_mul(a, b);
        } else {                  // a running sum of m terms (r_acc, r_settle), mixed scales
            const int m = 2 + (int)(rng() % 300);
            printf("%d ", m);
            R<L> acc = r_zero<L>();
            for (int q = 0; q < m; q++) {
                R<L> t = rand_r<L>(std::ldexp(1.0, (int)(rng() % 24) - 12));
                if (q > 0 && rng() % 4 == 0) t = r_neg(acc);  // cancel the sum so far
                if (q > 0 && rng() % 7 == 0) t = r_add(r_neg(acc), rand_r<L>(0x1p-60));
                acc = r_acc<L>(acc, t);
                out(t);
            }
            out(r_settle<L>(acc));
            printf("\n");
            continue;
        }
        out(a); out(b); out(r); printf("\n");
    }
}
int main(int argc, char **argv)
{
    const int L = atoi(argv[1]), mode = atoi(argv[2]), count = atoi(argv[3]);
    if (L == 2) run<2>(mode, count); else run<4>(mode, count);
    return 0;
}
