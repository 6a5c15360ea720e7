// Host-side check of the library's FP64-free arithmetic helpers (fx.cuh)
// against long double on random inputs.
#include "../paper_1006_0720_gb300/csrc/fx.cuh"
#include <cstdio>
#include <cmath>
#include <random>
#include <cstring>
static uint64_t dbits(double d){uint64_t u; memcpy(&u,&d,8); return u;}
static double bitsd(uint64_t u){double d; memcpy(&d,&u,8); return d;}
int main(){
  std::mt19937_64 g(1); int bad=0;
  std::uniform_real_distribution<double> U(-60,60);
  for(int i=0;i<2000000;i++){
    double x = U(g) * std::pow(2.0, -(int)(g()%40));
    int64_t X = fx::d2fix(dbits(x),56);
    long double ex = (long double)x * ldexpl(1.0L,56);
    if (fabsl((long double)X - ex) > 0.5000001L) { if(bad<5) printf("d2fix %.17g %lld %Lf\n",x,(long long)X,ex); bad++; }
    double back = bitsd(fx::fix2d(X,56));
    // fix2d must be RNE of X*2^-56
    long double exact = ldexpl((long double)X,-56);
    double rne = (double)exact;  // long double -> double is RNE
    if (back != rne) { if(bad<5) printf("fix2d %.17g %.17g\n",back,rne); bad++; }
    fx::df d = fx::fix2df(X,56);
    long double s = (long double)d.h + (long double)d.l;
    if (fabsl(s - exact) > fabsl(exact)*ldexpl(1.0L,-46) + ldexpl(1.0L,-60)) { if(bad<5) printf("fix2df %.17g\n",x); bad++; }
    fx::df e = fx::d2df(dbits(x));
    long double s2 = (long double)e.h + (long double)e.l;
    if (fabsl(s2 - (long double)x) > fabsl((long double)x)*ldexpl(1.0L,-46)) { if(bad<5) printf("d2df %.17g %.9g %.9g\n",x,e.h,e.l); bad++; }
    float f = (float)(U(g)*std::pow(2.0, -(int)(g()%30)));
    int64_t F = fx::f2fix(f,56);
    long double ef = (long double)f * ldexpl(1.0L,56);
    if (fabsl((long double)F - ef) > 0.5000001L) { if(bad<5) printf("f2fix %.9g\n",f); bad++; }
    // products and sums
    double a = U(g), b = U(g)*1e-3;
    fx::df da = fx::d2df(dbits(a)), db = fx::d2df(dbits(b));
    fx::df p = fx::df_norm(fx::mul(da,db));
    long double pe = (long double)a*(long double)b;
    if (fabsl(((long double)p.h+p.l) - pe) > fabsl(pe)*ldexpl(1.0L,-44)) { if(bad<5) printf("mul %.17g %.17g\n",a,b); bad++; }
    fx::df q = fx::add(da, db);
    long double qe = (long double)a + (long double)b;
    if (fabsl(((long double)q.h+q.l) - qe) > (fabsl((long double)a)+fabsl((long double)b))*ldexpl(1.0L,-45) + 1e-30L) { if(bad<5) printf("add %.17g %.17g\n",a,b); bad++; }
    double c = fabs(U(g)) + 1e-6;
    fx::df r = fx::sqrt_df(fx::d2df(dbits(c)));
    long double re = sqrtl((long double)c);
    if (fabsl(((long double)r.h+r.l) - re) > re*ldexpl(1.0L,-44)) { if(bad<5) printf("sqrt %.17g\n",c); bad++; }
  }
  // 128-bit integer -> double-float, reciprocals, double-float -> double
  for (int i = 0; i < 200000; i++) {
    __int128 v = ((__int128)(int64_t)g() << 40) ^ (__int128)(g() >> (g() % 64));
    if (g() & 1) v = -v;
    int sc = -(int)(g() % 100);
    fx::df d = fx::i128_to_df((uint64_t)v, (int64_t)(v >> 64), sc);
    long double ex = ldexpl((long double)v, sc);
    if (fabsl(((long double)d.h + d.l) - ex) > fabsl(ex) * ldexpl(1.0L, -45)) { if (bad < 5) printf("i128_to_df\n"); bad++; }
    int n = 1 + (int)(g() % 100000);
    fx::df r = fx::recip_df(n);
    if (fabsl(((long double)r.h + r.l) - 1.0L / n) > ldexpl(1.0L, -45) / n) { if (bad < 5) printf("recip %d\n", n); bad++; }
    double x = U(g) * std::pow(2.0, -(int)(g() % 60));
    fx::df dx = fx::d2df(dbits(x));
    double back = bitsd(fx::df2d(dx));
    long double sx = (long double)dx.h + (long double)dx.l;
    if (fabsl((long double)back - sx) > fabsl(sx) * ldexpl(1.0L, -52)) { if (bad < 5) printf("df2d %.17g\n", x); bad++; }
  }
  // FP64 -> double-float near the bottom of its range (2^-101 .. 2^-60),
  // where the low part leaves the FP32 normal range: a valid pair within
  // 2^-46 relative or 2^-125 absolute, and 0 below 2^-100
  for (int i = 0; i < 200000; i++) {
    const double x = (1.0 + U(g)) * std::pow(2.0, -60 - (int)(g() % 42)) * ((g() & 1) ? 1.0 : -1.0);
    const fx::df d = fx::d2df(dbits(x));
    const long double s = (long double)d.h + (long double)d.l;
    const bool finite = std::isfinite(d.h) && std::isfinite(d.l) && fabsl((long double)d.l) <= fabsl((long double)d.h);
    const long double tol = fabsl((long double)x) < ldexpl(1.0L, -100) ? fabsl((long double)x)
                                                                       : fabsl((long double)x) * ldexpl(1.0L, -46) + ldexpl(1.0L, -125);
    if (!finite || fabsl(s - (long double)x) > tol) {
      if (bad < 5) printf("d2df small %.17g -> %.9g %.9g\n", x, d.h, d.l);
      bad++;
    }
  }
  // FP64-free conversions: bit-identical to from_double / to_double on
  // doubles of every magnitude, exact floats, ties of the FP32 rounding and
  // arbitrary (also unnormalized) pairs
  std::uniform_real_distribution<double> U01(0.0, 1.0);
  for (int i = 0; i < 2000000; i++) {
    double x;
    const int kind = (int)(g() % 6);
    const double sgn = (g() & 1) ? 1.0 : -1.0;
    if (kind == 0) x = sgn * (1.0 + U01(g)) * std::pow(2.0, (int)(g() % 260) - 130);
    else if (kind == 1) x = sgn * (double)(float)(U01(g) * std::pow(2.0, (int)(g() % 60) - 30));
    else if (kind == 2) {  // a float plus exactly half its ulp (a tie), or a quarter
      const float f = (float)(1.0 + U01(g)) * (float)std::pow(2.0, (int)(g() % 40) - 20);
      x = sgn * ((double)f + std::ldexp(1.0, (int)((fx::f_bits(f) >> 23) & 0xFF) - 127 - 24 - (int)(g() % 2)));
    } else if (kind == 3) x = sgn * ldexp(1.0 + U01(g), -(int)(g() % 80));
    else if (kind == 4) x = sgn * ((double)(float)U01(g) + ldexp(U01(g), -(int)(30 + g() % 40)));
    else x = 0.0;
    uint64_t xb;
    memcpy(&xb, &x, 8);
    const fx::df a = fx::from_double(x), b = fx::d2df_rn(xb);
    if (fx::f_bits(a.h) != fx::f_bits(b.h) || fx::f_bits(a.l) != fx::f_bits(b.l)) {
      if (bad < 5) printf("d2df_rn %.17g: %.9g %.9g vs %.9g %.9g\n", x, a.h, a.l, b.h, b.l);
      bad++;
    }
    const double back = fx::to_double(a);
    uint64_t bb;
    memcpy(&bb, &back, 8);
    if (fx::df2d_rn(a) != bb) {
      if (bad < 5) printf("df2d_rn %.17g\n", x);
      bad++;
    }
    // FP32 -> FP64 bits
    const float fl = (float)(sgn * U01(g) * std::pow(2.0, (int)(g() % 300) - 150));
    const double fd = (double)fl;
    uint64_t fdb;
    memcpy(&fdb, &fd, 8);
    if (fx::f2d_bits(fl) != fdb) {
      if (bad < 5) printf("f2d_bits %.9g\n", fl);
      bad++;
    }
    // arbitrary pairs (the low part of any size and sign)
    const fx::df c = {(float)(sgn * (1.0 + U01(g)) * std::pow(2.0, (int)(g() % 200) - 100)),
                      (float)(((g() & 1) ? 1.0 : -1.0) * (1.0 + U01(g)) * std::pow(2.0, (int)(g() % 200) - 100))};
    const double cs = fx::to_double(c);
    uint64_t cb;
    memcpy(&cb, &cs, 8);
    if (fx::df2d_rn(c) != cb) {
      if (bad < 5) printf("df2d_rn pair %.9g %.9g\n", c.h, c.l);
      bad++;
    }
  }
  printf("bad %d\n", bad);
  return bad != 0;
}
