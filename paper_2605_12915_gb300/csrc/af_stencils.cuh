// GENERATED by gen_stencils.py -- do not edit.
// Exact frozen acoustic operator (Sec. 3.1; Appendix D compact monomial block)
// as orbit-compressed nodal stencils on the half-cell lattice around a node.
// L(dx, dy) returns the node values (.p, .u, .v) at lattice offset (dx, dy)
// in half cells; pK, uK, vK are the node's own values.  Accumulates, for
// r^1..r^4, Gp[o][q-1] (input p) and Guv[o][q-1] (inputs u, v), o = (pi,u,v).
#pragma once

// operation counts per node:
//   V : 184 multiply-adds, 128 adds
//   EV:  86 multiply-adds,  72 adds
//   EH:  86 multiply-adds,  72 adds
//   C :  27 multiply-adds,  40 adds

// family V: 8 orbit representatives
template <typename T, typename Load>
__device__ __forceinline__ void af_sac_V(const Load& L, T pK, T uK, T vK, T Gp[3][4], T Guv[3][4]) {
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int q = 0; q < 4; ++q) { Gp[o][q] = T(0); Guv[o][q] = T(0); }
  {  // orbit (+-0, +-1) half cells
    const auto n0 = L(0, 1);
    const auto n1 = L(0, -1);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][0] = fma(T(2.0), eep, Gp[0][0]);
    Gp[0][1] = fma(T(-5.81971863420548805845), eep, Gp[0][1]);
    Gp[0][2] = fma(T(5.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-2.0), eov, Guv[0][0]);
    Guv[0][1] = fma(T(5.0), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-3.87981242280365870564), eov, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), eov, Guv[0][3]);
    Guv[1][1] = fma(T(-1.90985931710274402923), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(2.33333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(-2.0), eop, Gp[2][0]);
    Gp[2][1] = fma(T(5.0), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-3.87981242280365870564), eop, Gp[2][2]);
    Gp[2][3] = fma(T(1.0), eop, Gp[2][3]);
    Guv[2][0] = fma(T(2.0), eev, Guv[2][0]);
    Guv[2][1] = fma(T(-3.90985931710274402923), eev, Guv[2][1]);
    Guv[2][2] = fma(T(2.66666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-0, +-2) half cells
    const auto n0 = L(0, 2);
    const auto n1 = L(0, -2);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][0] = fma(T(-0.5), eep, Gp[0][0]);
    Gp[0][1] = fma(T(1.95492965855137201461), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-2.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(0.5), eov, Guv[0][0]);
    Guv[0][1] = fma(T(-1.75), eov, Guv[0][1]);
    Guv[0][2] = fma(T(1.60657287806849601948), eov, Guv[0][2]);
    Guv[0][3] = fma(T(-0.5), eov, Guv[0][3]);
    Guv[1][1] = fma(T(0.477464829275686007307), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-0.833333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.333333333333333333333), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(0.5), eop, Gp[2][0]);
    Gp[2][1] = fma(T(-1.75), eop, Gp[2][1]);
    Gp[2][2] = fma(T(1.60657287806849601948), eop, Gp[2][2]);
    Gp[2][3] = fma(T(-0.5), eop, Gp[2][3]);
    Guv[2][0] = fma(T(-0.5), eev, Guv[2][0]);
    Guv[2][1] = fma(T(1.47746482927568600731), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-1.16666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.333333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-0) half cells
    const auto n0 = L(1, 0);
    const auto n1 = L(-1, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][0] = fma(T(2.0), eep, Gp[0][0]);
    Gp[0][1] = fma(T(-5.81971863420548805845), eep, Gp[0][1]);
    Gp[0][2] = fma(T(5.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-2.0), oeu, Guv[0][0]);
    Guv[0][1] = fma(T(5.0), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-3.87981242280365870564), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), oeu, Guv[0][3]);
    Gp[1][0] = fma(T(-2.0), oep, Gp[1][0]);
    Gp[1][1] = fma(T(5.0), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-3.87981242280365870564), oep, Gp[1][2]);
    Gp[1][3] = fma(T(1.0), oep, Gp[1][3]);
    Guv[1][0] = fma(T(2.0), eeu, Guv[1][0]);
    Guv[1][1] = fma(T(-3.90985931710274402923), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(2.66666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Guv[2][1] = fma(T(-1.90985931710274402923), eev, Guv[2][1]);
    Guv[2][2] = fma(T(2.33333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-1) half cells
    const auto n0 = L(1, 1);
    const auto n1 = L(1, -1);
    const auto n2 = L(-1, 1);
    const auto n3 = L(-1, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][1] = fma(T(2.5464790894703253723), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-4.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][1] = fma(T(-2.0), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(3.03098605964688358153), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(-1.0), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(-2.0), eov, Guv[0][1]);
    Guv[0][2] = fma(T(3.03098605964688358153), eov, Guv[0][2]);
    Guv[0][3] = fma(T(-1.0), eov, Guv[0][3]);
    Gp[1][1] = fma(T(-2.0), oep, Gp[1][1]);
    Gp[1][2] = fma(T(3.03098605964688358153), oep, Gp[1][2]);
    Gp[1][3] = fma(T(-1.0), oep, Gp[1][3]);
    Guv[1][1] = fma(T(1.27323954473516268615), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-2.0), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.666666666666666666667), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(2.0), oov, Guv[1][1]);
    Guv[1][2] = fma(T(-2.66666666666666666667), oov, Guv[1][2]);
    Guv[1][3] = fma(T(0.848826363156775124101), oov, Guv[1][3]);
    Gp[2][1] = fma(T(-2.0), eop, Gp[2][1]);
    Gp[2][2] = fma(T(3.03098605964688358153), eop, Gp[2][2]);
    Gp[2][3] = fma(T(-1.0), eop, Gp[2][3]);
    Guv[2][1] = fma(T(2.0), oou, Guv[2][1]);
    Guv[2][2] = fma(T(-2.66666666666666666667), oou, Guv[2][2]);
    Guv[2][3] = fma(T(0.848826363156775124101), oou, Guv[2][3]);
    Guv[2][1] = fma(T(1.27323954473516268615), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-2.0), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-2) half cells
    const auto n0 = L(1, 2);
    const auto n1 = L(1, -2);
    const auto n2 = L(-1, 2);
    const auto n3 = L(-1, -2);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][1] = fma(T(-0.636619772367581343076), eep, Gp[0][1]);
    Gp[0][2] = fma(T(1.5), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][1] = fma(T(0.5), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-1.09107984824505422872), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(0.5), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(0.5), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-1.18215969649010845743), eov, Guv[0][2]);
    Guv[0][3] = fma(T(0.5), eov, Guv[0][3]);
    Gp[1][1] = fma(T(0.5), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-1.09107984824505422872), oep, Gp[1][2]);
    Gp[1][3] = fma(T(0.5), oep, Gp[1][3]);
    Guv[1][1] = fma(T(-0.318309886183790671538), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(0.666666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.333333333333333333333), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(-0.5), oov, Guv[1][1]);
    Guv[1][2] = fma(T(1.0), oov, Guv[1][2]);
    Guv[1][3] = fma(T(-0.42441318157838756205), oov, Guv[1][3]);
    Gp[2][1] = fma(T(0.5), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-1.18215969649010845743), eop, Gp[2][2]);
    Gp[2][3] = fma(T(0.5), eop, Gp[2][3]);
    Guv[2][1] = fma(T(-0.5), oou, Guv[2][1]);
    Guv[2][2] = fma(T(1.0), oou, Guv[2][2]);
    Guv[2][3] = fma(T(-0.42441318157838756205), oou, Guv[2][3]);
    Guv[2][1] = fma(T(-0.318309886183790671538), eev, Guv[2][1]);
    Guv[2][2] = fma(T(0.833333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.333333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-2, +-0) half cells
    const auto n0 = L(2, 0);
    const auto n1 = L(-2, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][0] = fma(T(-0.5), eep, Gp[0][0]);
    Gp[0][1] = fma(T(1.95492965855137201461), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-2.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(0.5), oeu, Guv[0][0]);
    Guv[0][1] = fma(T(-1.75), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(1.60657287806849601948), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(-0.5), oeu, Guv[0][3]);
    Gp[1][0] = fma(T(0.5), oep, Gp[1][0]);
    Gp[1][1] = fma(T(-1.75), oep, Gp[1][1]);
    Gp[1][2] = fma(T(1.60657287806849601948), oep, Gp[1][2]);
    Gp[1][3] = fma(T(-0.5), oep, Gp[1][3]);
    Guv[1][0] = fma(T(-0.5), eeu, Guv[1][0]);
    Guv[1][1] = fma(T(1.47746482927568600731), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-1.16666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.333333333333333333333), eeu, Guv[1][3]);
    Guv[2][1] = fma(T(0.477464829275686007307), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-0.833333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.333333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-2, +-1) half cells
    const auto n0 = L(2, 1);
    const auto n1 = L(2, -1);
    const auto n2 = L(-2, 1);
    const auto n3 = L(-2, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][1] = fma(T(-0.636619772367581343076), eep, Gp[0][1]);
    Gp[0][2] = fma(T(1.5), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][1] = fma(T(0.5), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-1.18215969649010845743), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(0.5), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(0.5), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-1.09107984824505422872), eov, Guv[0][2]);
    Guv[0][3] = fma(T(0.5), eov, Guv[0][3]);
    Gp[1][1] = fma(T(0.5), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-1.18215969649010845743), oep, Gp[1][2]);
    Gp[1][3] = fma(T(0.5), oep, Gp[1][3]);
    Guv[1][1] = fma(T(-0.318309886183790671538), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(0.833333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.333333333333333333333), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(-0.5), oov, Guv[1][1]);
    Guv[1][2] = fma(T(1.0), oov, Guv[1][2]);
    Guv[1][3] = fma(T(-0.42441318157838756205), oov, Guv[1][3]);
    Gp[2][1] = fma(T(0.5), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-1.09107984824505422872), eop, Gp[2][2]);
    Gp[2][3] = fma(T(0.5), eop, Gp[2][3]);
    Guv[2][1] = fma(T(-0.5), oou, Guv[2][1]);
    Guv[2][2] = fma(T(1.0), oou, Guv[2][2]);
    Guv[2][3] = fma(T(-0.42441318157838756205), oou, Guv[2][3]);
    Guv[2][1] = fma(T(-0.318309886183790671538), eev, Guv[2][1]);
    Guv[2][2] = fma(T(0.666666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.333333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-2, +-2) half cells
    const auto n0 = L(2, 2);
    const auto n1 = L(2, -2);
    const auto n2 = L(-2, 2);
    const auto n3 = L(-2, -2);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][1] = fma(T(0.159154943091895335769), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-0.5), eep, Gp[0][2]);
    Gp[0][3] = fma(T(0.333333333333333333333), eep, Gp[0][3]);
    Guv[0][1] = fma(T(-0.125), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(0.378873257455860447692), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(-0.25), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(-0.125), eov, Guv[0][1]);
    Guv[0][2] = fma(T(0.378873257455860447692), eov, Guv[0][2]);
    Guv[0][3] = fma(T(-0.25), eov, Guv[0][3]);
    Gp[1][1] = fma(T(-0.125), oep, Gp[1][1]);
    Gp[1][2] = fma(T(0.378873257455860447692), oep, Gp[1][2]);
    Gp[1][3] = fma(T(-0.25), oep, Gp[1][3]);
    Guv[1][1] = fma(T(0.0795774715459476678844), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-0.25), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.166666666666666666667), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(0.125), oov, Guv[1][1]);
    Guv[1][2] = fma(T(-0.333333333333333333333), oov, Guv[1][2]);
    Guv[1][3] = fma(T(0.212206590789193781025), oov, Guv[1][3]);
    Gp[2][1] = fma(T(-0.125), eop, Gp[2][1]);
    Gp[2][2] = fma(T(0.378873257455860447692), eop, Gp[2][2]);
    Gp[2][3] = fma(T(-0.25), eop, Gp[2][3]);
    Guv[2][1] = fma(T(0.125), oou, Guv[2][1]);
    Guv[2][2] = fma(T(-0.333333333333333333333), oou, Guv[2][2]);
    Guv[2][3] = fma(T(0.212206590789193781025), oou, Guv[2][3]);
    Guv[2][1] = fma(T(0.0795774715459476678844), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-0.25), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.166666666666666666667), eev, Guv[2][3]);
  }
}

// family EV: 5 orbit representatives
template <typename T, typename Load>
__device__ __forceinline__ void af_sac_EV(const Load& L, T pK, T uK, T vK, T Gp[3][4], T Guv[3][4]) {
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int q = 0; q < 4; ++q) { Gp[o][q] = T(0); Guv[o][q] = T(0); }
  {  // orbit (+-0, +-1) half cells
    const auto n0 = L(0, 1);
    const auto n1 = L(0, -1);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][1] = fma(T(2.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-3.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-1.0), eov, Guv[0][0]);
    Guv[0][1] = fma(T(1.5), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-0.666666666666666666667), eov, Guv[0][2]);
    Guv[1][2] = fma(T(-1.0), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.666666666666666666667), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(-1.0), eop, Gp[2][0]);
    Gp[2][1] = fma(T(1.5), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-0.666666666666666666667), eop, Gp[2][2]);
    Guv[2][1] = fma(T(2.0), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-2.0), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-0) half cells
    const auto n0 = L(1, 0);
    const auto n1 = L(-1, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][0] = fma(T(2.0), eep, Gp[0][0]);
    Gp[0][1] = fma(T(-2.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-4.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(2.66666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-2.0), oeu, Guv[0][0]);
    Guv[0][1] = fma(T(2.0), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(2.66666666666666666667), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(-2.0), oeu, Guv[0][3]);
    Gp[1][0] = fma(T(-2.0), oep, Gp[1][0]);
    Gp[1][1] = fma(T(2.0), oep, Gp[1][1]);
    Gp[1][2] = fma(T(2.66666666666666666667), oep, Gp[1][2]);
    Gp[1][3] = fma(T(-2.0), oep, Gp[1][3]);
    Guv[1][0] = fma(T(2.0), eeu, Guv[1][0]);
    Guv[1][1] = fma(T(-2.0), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-1.33333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(1.33333333333333333333), eeu, Guv[1][3]);
    Guv[2][2] = fma(T(-2.66666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(1.33333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-1) half cells
    const auto n0 = L(1, 1);
    const auto n1 = L(1, -1);
    const auto n2 = L(-1, 1);
    const auto n3 = L(-1, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][2] = fma(T(2.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][2] = fma(T(-1.33333333333333333333), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(-1.0), eov, Guv[0][1]);
    Guv[0][2] = fma(T(0.666666666666666666667), eov, Guv[0][2]);
    Gp[1][2] = fma(T(-1.33333333333333333333), oep, Gp[1][2]);
    Gp[1][3] = fma(T(1.0), oep, Gp[1][3]);
    Guv[1][2] = fma(T(0.666666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(1.0), oov, Guv[1][1]);
    Guv[1][2] = fma(T(-0.666666666666666666667), oov, Guv[1][2]);
    Gp[2][1] = fma(T(-1.0), eop, Gp[2][1]);
    Gp[2][2] = fma(T(0.666666666666666666667), eop, Gp[2][2]);
    Guv[2][1] = fma(T(1.0), oou, Guv[2][1]);
    Guv[2][2] = fma(T(-0.666666666666666666667), oou, Guv[2][2]);
    Guv[2][2] = fma(T(1.33333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-2, +-0) half cells
    const auto n0 = L(2, 0);
    const auto n1 = L(-2, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][0] = fma(T(-0.5), eep, Gp[0][0]);
    Gp[0][1] = fma(T(1.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(1.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(0.5), oeu, Guv[0][0]);
    Guv[0][1] = fma(T(-1.0), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-0.666666666666666666667), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), oeu, Guv[0][3]);
    Gp[1][0] = fma(T(0.5), oep, Gp[1][0]);
    Gp[1][1] = fma(T(-1.0), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-0.666666666666666666667), oep, Gp[1][2]);
    Gp[1][3] = fma(T(1.0), oep, Gp[1][3]);
    Guv[1][0] = fma(T(-0.5), eeu, Guv[1][0]);
    Guv[1][1] = fma(T(1.0), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(0.333333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Guv[2][2] = fma(T(0.666666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-2, +-1) half cells
    const auto n0 = L(2, 1);
    const auto n1 = L(2, -1);
    const auto n2 = L(-2, 1);
    const auto n3 = L(-2, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][2] = fma(T(-0.5), eep, Gp[0][2]);
    Gp[0][3] = fma(T(0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][2] = fma(T(0.333333333333333333333), oeu, Guv[0][2]);
    Guv[0][3] = fma(T(-0.5), oeu, Guv[0][3]);
    Guv[0][1] = fma(T(0.25), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-0.333333333333333333333), eov, Guv[0][2]);
    Gp[1][2] = fma(T(0.333333333333333333333), oep, Gp[1][2]);
    Gp[1][3] = fma(T(-0.5), oep, Gp[1][3]);
    Guv[1][2] = fma(T(-0.166666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.333333333333333333333), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(-0.25), oov, Guv[1][1]);
    Guv[1][2] = fma(T(0.333333333333333333333), oov, Guv[1][2]);
    Gp[2][1] = fma(T(0.25), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-0.333333333333333333333), eop, Gp[2][2]);
    Guv[2][1] = fma(T(-0.25), oou, Guv[2][1]);
    Guv[2][2] = fma(T(0.333333333333333333333), oou, Guv[2][2]);
    Guv[2][2] = fma(T(-0.333333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.333333333333333333333), eev, Guv[2][3]);
  }
}

// family EH: 5 orbit representatives
template <typename T, typename Load>
__device__ __forceinline__ void af_sac_EH(const Load& L, T pK, T uK, T vK, T Gp[3][4], T Guv[3][4]) {
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int q = 0; q < 4; ++q) { Gp[o][q] = T(0); Guv[o][q] = T(0); }
  {  // orbit (+-0, +-1) half cells
    const auto n0 = L(0, 1);
    const auto n1 = L(0, -1);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][0] = fma(T(2.0), eep, Gp[0][0]);
    Gp[0][1] = fma(T(-2.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-4.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(2.66666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-2.0), eov, Guv[0][0]);
    Guv[0][1] = fma(T(2.0), eov, Guv[0][1]);
    Guv[0][2] = fma(T(2.66666666666666666667), eov, Guv[0][2]);
    Guv[0][3] = fma(T(-2.0), eov, Guv[0][3]);
    Guv[1][2] = fma(T(-2.66666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(1.33333333333333333333), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(-2.0), eop, Gp[2][0]);
    Gp[2][1] = fma(T(2.0), eop, Gp[2][1]);
    Gp[2][2] = fma(T(2.66666666666666666667), eop, Gp[2][2]);
    Gp[2][3] = fma(T(-2.0), eop, Gp[2][3]);
    Guv[2][0] = fma(T(2.0), eev, Guv[2][0]);
    Guv[2][1] = fma(T(-2.0), eev, Guv[2][1]);
    Guv[2][2] = fma(T(-1.33333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(1.33333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-0, +-2) half cells
    const auto n0 = L(0, 2);
    const auto n1 = L(0, -2);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][0] = fma(T(-0.5), eep, Gp[0][0]);
    Gp[0][1] = fma(T(1.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(1.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(0.5), eov, Guv[0][0]);
    Guv[0][1] = fma(T(-1.0), eov, Guv[0][1]);
    Guv[0][2] = fma(T(-0.666666666666666666667), eov, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), eov, Guv[0][3]);
    Guv[1][2] = fma(T(0.666666666666666666667), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(0.5), eop, Gp[2][0]);
    Gp[2][1] = fma(T(-1.0), eop, Gp[2][1]);
    Gp[2][2] = fma(T(-0.666666666666666666667), eop, Gp[2][2]);
    Gp[2][3] = fma(T(1.0), eop, Gp[2][3]);
    Guv[2][0] = fma(T(-0.5), eev, Guv[2][0]);
    Guv[2][1] = fma(T(1.0), eev, Guv[2][1]);
    Guv[2][2] = fma(T(0.333333333333333333333), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-0) half cells
    const auto n0 = L(1, 0);
    const auto n1 = L(-1, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][1] = fma(T(2.0), eep, Gp[0][1]);
    Gp[0][2] = fma(T(-3.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-1.0), oeu, Guv[0][0]);
    Guv[0][1] = fma(T(1.5), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-0.666666666666666666667), oeu, Guv[0][2]);
    Gp[1][0] = fma(T(-1.0), oep, Gp[1][0]);
    Gp[1][1] = fma(T(1.5), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-0.666666666666666666667), oep, Gp[1][2]);
    Guv[1][1] = fma(T(2.0), eeu, Guv[1][1]);
    Guv[1][2] = fma(T(-2.0), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.666666666666666666667), eeu, Guv[1][3]);
    Guv[2][2] = fma(T(-1.0), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-1) half cells
    const auto n0 = L(1, 1);
    const auto n1 = L(1, -1);
    const auto n2 = L(-1, 1);
    const auto n3 = L(-1, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][2] = fma(T(2.0), eep, Gp[0][2]);
    Gp[0][3] = fma(T(-1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][1] = fma(T(-1.0), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(0.666666666666666666667), oeu, Guv[0][2]);
    Guv[0][2] = fma(T(-1.33333333333333333333), eov, Guv[0][2]);
    Guv[0][3] = fma(T(1.0), eov, Guv[0][3]);
    Gp[1][1] = fma(T(-1.0), oep, Gp[1][1]);
    Gp[1][2] = fma(T(0.666666666666666666667), oep, Gp[1][2]);
    Guv[1][2] = fma(T(1.33333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(-0.666666666666666666667), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(1.0), oov, Guv[1][1]);
    Guv[1][2] = fma(T(-0.666666666666666666667), oov, Guv[1][2]);
    Gp[2][2] = fma(T(-1.33333333333333333333), eop, Gp[2][2]);
    Gp[2][3] = fma(T(1.0), eop, Gp[2][3]);
    Guv[2][1] = fma(T(1.0), oou, Guv[2][1]);
    Guv[2][2] = fma(T(-0.666666666666666666667), oou, Guv[2][2]);
    Guv[2][2] = fma(T(0.666666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(-0.666666666666666666667), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-2) half cells
    const auto n0 = L(1, 2);
    const auto n1 = L(1, -2);
    const auto n2 = L(-1, 2);
    const auto n3 = L(-1, -2);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][2] = fma(T(-0.5), eep, Gp[0][2]);
    Gp[0][3] = fma(T(0.666666666666666666667), eep, Gp[0][3]);
    Guv[0][1] = fma(T(0.25), oeu, Guv[0][1]);
    Guv[0][2] = fma(T(-0.333333333333333333333), oeu, Guv[0][2]);
    Guv[0][2] = fma(T(0.333333333333333333333), eov, Guv[0][2]);
    Guv[0][3] = fma(T(-0.5), eov, Guv[0][3]);
    Gp[1][1] = fma(T(0.25), oep, Gp[1][1]);
    Gp[1][2] = fma(T(-0.333333333333333333333), oep, Gp[1][2]);
    Guv[1][2] = fma(T(-0.333333333333333333333), eeu, Guv[1][2]);
    Guv[1][3] = fma(T(0.333333333333333333333), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(-0.25), oov, Guv[1][1]);
    Guv[1][2] = fma(T(0.333333333333333333333), oov, Guv[1][2]);
    Gp[2][2] = fma(T(0.333333333333333333333), eop, Gp[2][2]);
    Gp[2][3] = fma(T(-0.5), eop, Gp[2][3]);
    Guv[2][1] = fma(T(-0.25), oou, Guv[2][1]);
    Guv[2][2] = fma(T(0.333333333333333333333), oou, Guv[2][2]);
    Guv[2][2] = fma(T(-0.166666666666666666667), eev, Guv[2][2]);
    Guv[2][3] = fma(T(0.333333333333333333333), eev, Guv[2][3]);
  }
}

// family C: 3 orbit representatives
template <typename T, typename Load>
__device__ __forceinline__ void af_sac_C(const Load& L, T pK, T uK, T vK, T Gp[3][4], T Guv[3][4]) {
#pragma unroll
  for (int o = 0; o < 3; ++o)
#pragma unroll
    for (int q = 0; q < 4; ++q) { Gp[o][q] = T(0); Guv[o][q] = T(0); }
  {  // orbit (+-0, +-1) half cells
    const auto n0 = L(0, 1);
    const auto n1 = L(0, -1);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T eop = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    const T eov = n0.v - n1.v;
    Gp[0][1] = fma(T(2.0), eep, Gp[0][1]);
    Gp[0][3] = fma(T(-2.66666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-1.0), eov, Guv[0][0]);
    Guv[0][2] = fma(T(1.33333333333333333333), eov, Guv[0][2]);
    Guv[1][3] = fma(T(-1.33333333333333333333), eeu, Guv[1][3]);
    Gp[2][0] = fma(T(-1.0), eop, Gp[2][0]);
    Gp[2][2] = fma(T(1.33333333333333333333), eop, Gp[2][2]);
    Guv[2][1] = fma(T(2.0), eev, Guv[2][1]);
    Guv[2][3] = fma(T(-1.33333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-0) half cells
    const auto n0 = L(1, 0);
    const auto n1 = L(-1, 0);
    const T eep = (n0.p + n1.p) - T(2) * pK;
    const T oep = n0.p - n1.p;
    const T eeu = (n0.u + n1.u) - T(2) * uK;
    const T oeu = n0.u - n1.u;
    const T eev = (n0.v + n1.v) - T(2) * vK;
    Gp[0][1] = fma(T(2.0), eep, Gp[0][1]);
    Gp[0][3] = fma(T(-2.66666666666666666667), eep, Gp[0][3]);
    Guv[0][0] = fma(T(-1.0), oeu, Guv[0][0]);
    Guv[0][2] = fma(T(1.33333333333333333333), oeu, Guv[0][2]);
    Gp[1][0] = fma(T(-1.0), oep, Gp[1][0]);
    Gp[1][2] = fma(T(1.33333333333333333333), oep, Gp[1][2]);
    Guv[1][1] = fma(T(2.0), eeu, Guv[1][1]);
    Guv[1][3] = fma(T(-1.33333333333333333333), eeu, Guv[1][3]);
    Guv[2][3] = fma(T(-1.33333333333333333333), eev, Guv[2][3]);
  }
  {  // orbit (+-1, +-1) half cells
    const auto n0 = L(1, 1);
    const auto n1 = L(1, -1);
    const auto n2 = L(-1, 1);
    const auto n3 = L(-1, -1);
    const T s12p = n0.p + n2.p, d12p = n0.p - n2.p;
    const T s34p = n1.p + n3.p, d34p = n1.p - n3.p;
    const T eep = (s12p + s34p) - T(4) * pK;
    const T eop = s12p - s34p;
    const T oep = d12p + d34p;
    const T s12u = n0.u + n2.u, d12u = n0.u - n2.u;
    const T s34u = n1.u + n3.u, d34u = n1.u - n3.u;
    const T eeu = (s12u + s34u) - T(4) * uK;
    const T oeu = d12u + d34u;
    const T oou = d12u - d34u;
    const T s12v = n0.v + n2.v, d12v = n0.v - n2.v;
    const T s34v = n1.v + n3.v, d34v = n1.v - n3.v;
    const T eev = (s12v + s34v) - T(4) * vK;
    const T eov = s12v - s34v;
    const T oov = d12v - d34v;
    Gp[0][3] = fma(T(1.33333333333333333333), eep, Gp[0][3]);
    Guv[0][2] = fma(T(-0.666666666666666666667), oeu, Guv[0][2]);
    Guv[0][2] = fma(T(-0.666666666666666666667), eov, Guv[0][2]);
    Gp[1][2] = fma(T(-0.666666666666666666667), oep, Gp[1][2]);
    Guv[1][3] = fma(T(0.666666666666666666667), eeu, Guv[1][3]);
    Guv[1][1] = fma(T(0.5), oov, Guv[1][1]);
    Gp[2][2] = fma(T(-0.666666666666666666667), eop, Gp[2][2]);
    Guv[2][1] = fma(T(0.5), oou, Guv[2][1]);
    Guv[2][3] = fma(T(0.666666666666666666667), eev, Guv[2][3]);
  }
}
