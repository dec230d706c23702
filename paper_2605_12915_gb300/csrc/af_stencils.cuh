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

// family V, transposed: lattice adjoints from output adjoints
template <typename T, typename Scatter>
__device__ __forceinline__ void af_sac_V_adj(const Scatter& S, const T lGp[3][4], const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  T c0m2[3];  // the values of member (0, -2), held for its triple
  T c0m1[3];  // the values of member (0, -1), held for its triple
  T c0p1[3];  // the values of member (0, 1), held for its triple
  T c0p2[3];  // the values of member (0, 2), held for its triple
  {  // orbit (+-0, +-1) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(5.0), lGp[0][2], fma(T(-5.81971863420548805845), lGp[0][1], fma(T(2.0), lGp[0][0], T(0)))));
    const T leop = fma(T(1.0), lGp[2][3], fma(T(-3.87981242280365870564), lGp[2][2], fma(T(5.0), lGp[2][1], fma(T(-2.0), lGp[2][0], T(0)))));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(2.33333333333333333333), lGuv[1][2], fma(T(-1.90985931710274402923), lGuv[1][1], T(0))));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(2.66666666666666666667), lGuv[2][2], fma(T(-3.90985931710274402923), lGuv[2][1], fma(T(2.0), lGuv[2][0], T(0)))));
    const T leov = fma(T(1.0), lGuv[0][3], fma(T(-3.87981242280365870564), lGuv[0][2], fma(T(5.0), lGuv[0][1], fma(T(-2.0), lGuv[0][0], T(0)))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    c0p1[0] = T(0) + leep + leop;
    c0p1[1] = T(0) + leeu;
    c0p1[2] = T(0) + leev + leov;
    c0m1[0] = T(0) + leep - leop;
    c0m1[1] = T(0) + leeu;
    c0m1[2] = T(0) + leev - leov;
  }
  {  // orbit (+-0, +-2) half cells
    const T leep = fma(T(0.666666666666666666667), lGp[0][3], fma(T(-2.0), lGp[0][2], fma(T(1.95492965855137201461), lGp[0][1], fma(T(-0.5), lGp[0][0], T(0)))));
    const T leop = fma(T(-0.5), lGp[2][3], fma(T(1.60657287806849601948), lGp[2][2], fma(T(-1.75), lGp[2][1], fma(T(0.5), lGp[2][0], T(0)))));
    const T leeu = fma(T(0.333333333333333333333), lGuv[1][3], fma(T(-0.833333333333333333333), lGuv[1][2], fma(T(0.477464829275686007307), lGuv[1][1], T(0))));
    const T leev = fma(T(0.333333333333333333333), lGuv[2][3], fma(T(-1.16666666666666666667), lGuv[2][2], fma(T(1.47746482927568600731), lGuv[2][1], fma(T(-0.5), lGuv[2][0], T(0)))));
    const T leov = fma(T(-0.5), lGuv[0][3], fma(T(1.60657287806849601948), lGuv[0][2], fma(T(-1.75), lGuv[0][1], fma(T(0.5), lGuv[0][0], T(0)))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    c0p2[0] = T(0) + leep + leop;
    c0p2[1] = T(0) + leeu;
    c0p2[2] = T(0) + leev + leov;
    c0m2[0] = T(0) + leep - leop;
    c0m2[1] = T(0) + leeu;
    c0m2[2] = T(0) + leev - leov;
  }
  {  // orbit (+-1, +-0) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(5.0), lGp[0][2], fma(T(-5.81971863420548805845), lGp[0][1], fma(T(2.0), lGp[0][0], T(0)))));
    const T loep = fma(T(1.0), lGp[1][3], fma(T(-3.87981242280365870564), lGp[1][2], fma(T(5.0), lGp[1][1], fma(T(-2.0), lGp[1][0], T(0)))));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(2.66666666666666666667), lGuv[1][2], fma(T(-3.90985931710274402923), lGuv[1][1], fma(T(2.0), lGuv[1][0], T(0)))));
    const T loeu = fma(T(1.0), lGuv[0][3], fma(T(-3.87981242280365870564), lGuv[0][2], fma(T(5.0), lGuv[0][1], fma(T(-2.0), lGuv[0][0], T(0)))));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(2.33333333333333333333), lGuv[2][2], fma(T(-1.90985931710274402923), lGuv[2][1], T(0))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(1, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-1, +-1) half cells
    const T leep = fma(T(1.33333333333333333333), lGp[0][3], fma(T(-4.0), lGp[0][2], fma(T(2.5464790894703253723), lGp[0][1], T(0))));
    const T loep = fma(T(-1.0), lGp[1][3], fma(T(3.03098605964688358153), lGp[1][2], fma(T(-2.0), lGp[1][1], T(0))));
    const T leop = fma(T(-1.0), lGp[2][3], fma(T(3.03098605964688358153), lGp[2][2], fma(T(-2.0), lGp[2][1], T(0))));
    const T leeu = fma(T(0.666666666666666666667), lGuv[1][3], fma(T(-2.0), lGuv[1][2], fma(T(1.27323954473516268615), lGuv[1][1], T(0))));
    const T loeu = fma(T(-1.0), lGuv[0][3], fma(T(3.03098605964688358153), lGuv[0][2], fma(T(-2.0), lGuv[0][1], T(0))));
    const T loou = fma(T(0.848826363156775124101), lGuv[2][3], fma(T(-2.66666666666666666667), lGuv[2][2], fma(T(2.0), lGuv[2][1], T(0))));
    const T leev = fma(T(0.666666666666666666667), lGuv[2][3], fma(T(-2.0), lGuv[2][2], fma(T(1.27323954473516268615), lGuv[2][1], T(0))));
    const T leov = fma(T(-1.0), lGuv[0][3], fma(T(3.03098605964688358153), lGuv[0][2], fma(T(-2.0), lGuv[0][1], T(0))));
    const T loov = fma(T(0.848826363156775124101), lGuv[1][3], fma(T(-2.66666666666666666667), lGuv[1][2], fma(T(2.0), lGuv[1][1], T(0))));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
  }
  {  // orbit (+-1, +-2) half cells
    const T leep = fma(T(-0.666666666666666666667), lGp[0][3], fma(T(1.5), lGp[0][2], fma(T(-0.636619772367581343076), lGp[0][1], T(0))));
    const T loep = fma(T(0.5), lGp[1][3], fma(T(-1.09107984824505422872), lGp[1][2], fma(T(0.5), lGp[1][1], T(0))));
    const T leop = fma(T(0.5), lGp[2][3], fma(T(-1.18215969649010845743), lGp[2][2], fma(T(0.5), lGp[2][1], T(0))));
    const T leeu = fma(T(-0.333333333333333333333), lGuv[1][3], fma(T(0.666666666666666666667), lGuv[1][2], fma(T(-0.318309886183790671538), lGuv[1][1], T(0))));
    const T loeu = fma(T(0.5), lGuv[0][3], fma(T(-1.09107984824505422872), lGuv[0][2], fma(T(0.5), lGuv[0][1], T(0))));
    const T loou = fma(T(-0.42441318157838756205), lGuv[2][3], fma(T(1.0), lGuv[2][2], fma(T(-0.5), lGuv[2][1], T(0))));
    const T leev = fma(T(-0.333333333333333333333), lGuv[2][3], fma(T(0.833333333333333333333), lGuv[2][2], fma(T(-0.318309886183790671538), lGuv[2][1], T(0))));
    const T leov = fma(T(0.5), lGuv[0][3], fma(T(-1.18215969649010845743), lGuv[0][2], fma(T(0.5), lGuv[0][1], T(0))));
    const T loov = fma(T(-0.42441318157838756205), lGuv[1][3], fma(T(1.0), lGuv[1][2], fma(T(-0.5), lGuv[1][1], T(0))));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 2, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -2, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
  }
  {  // orbit (+-2, +-0) half cells
    const T leep = fma(T(0.666666666666666666667), lGp[0][3], fma(T(-2.0), lGp[0][2], fma(T(1.95492965855137201461), lGp[0][1], fma(T(-0.5), lGp[0][0], T(0)))));
    const T loep = fma(T(-0.5), lGp[1][3], fma(T(1.60657287806849601948), lGp[1][2], fma(T(-1.75), lGp[1][1], fma(T(0.5), lGp[1][0], T(0)))));
    const T leeu = fma(T(0.333333333333333333333), lGuv[1][3], fma(T(-1.16666666666666666667), lGuv[1][2], fma(T(1.47746482927568600731), lGuv[1][1], fma(T(-0.5), lGuv[1][0], T(0)))));
    const T loeu = fma(T(-0.5), lGuv[0][3], fma(T(1.60657287806849601948), lGuv[0][2], fma(T(-1.75), lGuv[0][1], fma(T(0.5), lGuv[0][0], T(0)))));
    const T leev = fma(T(0.333333333333333333333), lGuv[2][3], fma(T(-0.833333333333333333333), lGuv[2][2], fma(T(0.477464829275686007307), lGuv[2][1], T(0))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(2, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-2, +-1) half cells
    const T leep = fma(T(-0.666666666666666666667), lGp[0][3], fma(T(1.5), lGp[0][2], fma(T(-0.636619772367581343076), lGp[0][1], T(0))));
    const T loep = fma(T(0.5), lGp[1][3], fma(T(-1.18215969649010845743), lGp[1][2], fma(T(0.5), lGp[1][1], T(0))));
    const T leop = fma(T(0.5), lGp[2][3], fma(T(-1.09107984824505422872), lGp[2][2], fma(T(0.5), lGp[2][1], T(0))));
    const T leeu = fma(T(-0.333333333333333333333), lGuv[1][3], fma(T(0.833333333333333333333), lGuv[1][2], fma(T(-0.318309886183790671538), lGuv[1][1], T(0))));
    const T loeu = fma(T(0.5), lGuv[0][3], fma(T(-1.18215969649010845743), lGuv[0][2], fma(T(0.5), lGuv[0][1], T(0))));
    const T loou = fma(T(-0.42441318157838756205), lGuv[2][3], fma(T(1.0), lGuv[2][2], fma(T(-0.5), lGuv[2][1], T(0))));
    const T leev = fma(T(-0.333333333333333333333), lGuv[2][3], fma(T(0.666666666666666666667), lGuv[2][2], fma(T(-0.318309886183790671538), lGuv[2][1], T(0))));
    const T leov = fma(T(0.5), lGuv[0][3], fma(T(-1.09107984824505422872), lGuv[0][2], fma(T(0.5), lGuv[0][1], T(0))));
    const T loov = fma(T(-0.42441318157838756205), lGuv[1][3], fma(T(1.0), lGuv[1][2], fma(T(-0.5), lGuv[1][1], T(0))));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.triple(1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
             T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov,
             c0p1[0], c0p1[1], c0p1[2]);
    S.triple(-1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
             T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov,
             c0m1[0], c0m1[1], c0m1[2]);
  }
  {  // orbit (+-2, +-2) half cells
    const T leep = fma(T(0.333333333333333333333), lGp[0][3], fma(T(-0.5), lGp[0][2], fma(T(0.159154943091895335769), lGp[0][1], T(0))));
    const T loep = fma(T(-0.25), lGp[1][3], fma(T(0.378873257455860447692), lGp[1][2], fma(T(-0.125), lGp[1][1], T(0))));
    const T leop = fma(T(-0.25), lGp[2][3], fma(T(0.378873257455860447692), lGp[2][2], fma(T(-0.125), lGp[2][1], T(0))));
    const T leeu = fma(T(0.166666666666666666667), lGuv[1][3], fma(T(-0.25), lGuv[1][2], fma(T(0.0795774715459476678844), lGuv[1][1], T(0))));
    const T loeu = fma(T(-0.25), lGuv[0][3], fma(T(0.378873257455860447692), lGuv[0][2], fma(T(-0.125), lGuv[0][1], T(0))));
    const T loou = fma(T(0.212206590789193781025), lGuv[2][3], fma(T(-0.333333333333333333333), lGuv[2][2], fma(T(0.125), lGuv[2][1], T(0))));
    const T leev = fma(T(0.166666666666666666667), lGuv[2][3], fma(T(-0.25), lGuv[2][2], fma(T(0.0795774715459476678844), lGuv[2][1], T(0))));
    const T leov = fma(T(-0.25), lGuv[0][3], fma(T(0.378873257455860447692), lGuv[0][2], fma(T(-0.125), lGuv[0][1], T(0))));
    const T loov = fma(T(0.212206590789193781025), lGuv[1][3], fma(T(-0.333333333333333333333), lGuv[1][2], fma(T(0.125), lGuv[1][1], T(0))));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.triple(2, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
             T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov,
             c0p2[0], c0p2[1], c0p2[2]);
    S.triple(-2, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
             T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov,
             c0m2[0], c0m2[1], c0m2[2]);
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

// family EV, transposed: lattice adjoints from output adjoints
template <typename T, typename Scatter>
__device__ __forceinline__ void af_sac_EV_adj(const Scatter& S, const T lGp[3][4], const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  T c0m1[3];  // the values of member (0, -1), held for its triple
  T c0p1[3];  // the values of member (0, 1), held for its triple
  {  // orbit (+-0, +-1) half cells
    const T leep = fma(T(1.33333333333333333333), lGp[0][3], fma(T(-3.0), lGp[0][2], fma(T(2.0), lGp[0][1], T(0))));
    const T leop = fma(T(-0.666666666666666666667), lGp[2][2], fma(T(1.5), lGp[2][1], fma(T(-1.0), lGp[2][0], T(0))));
    const T leeu = fma(T(0.666666666666666666667), lGuv[1][3], fma(T(-1.0), lGuv[1][2], T(0)));
    const T leev = fma(T(0.666666666666666666667), lGuv[2][3], fma(T(-2.0), lGuv[2][2], fma(T(2.0), lGuv[2][1], T(0))));
    const T leov = fma(T(-0.666666666666666666667), lGuv[0][2], fma(T(1.5), lGuv[0][1], fma(T(-1.0), lGuv[0][0], T(0))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    c0p1[0] = T(0) + leep + leop;
    c0p1[1] = T(0) + leeu;
    c0p1[2] = T(0) + leev + leov;
    c0m1[0] = T(0) + leep - leop;
    c0m1[1] = T(0) + leeu;
    c0m1[2] = T(0) + leev - leov;
  }
  {  // orbit (+-1, +-0) half cells
    const T leep = fma(T(2.66666666666666666667), lGp[0][3], fma(T(-4.0), lGp[0][2], fma(T(-2.0), lGp[0][1], fma(T(2.0), lGp[0][0], T(0)))));
    const T loep = fma(T(-2.0), lGp[1][3], fma(T(2.66666666666666666667), lGp[1][2], fma(T(2.0), lGp[1][1], fma(T(-2.0), lGp[1][0], T(0)))));
    const T leeu = fma(T(1.33333333333333333333), lGuv[1][3], fma(T(-1.33333333333333333333), lGuv[1][2], fma(T(-2.0), lGuv[1][1], fma(T(2.0), lGuv[1][0], T(0)))));
    const T loeu = fma(T(-2.0), lGuv[0][3], fma(T(2.66666666666666666667), lGuv[0][2], fma(T(2.0), lGuv[0][1], fma(T(-2.0), lGuv[0][0], T(0)))));
    const T leev = fma(T(1.33333333333333333333), lGuv[2][3], fma(T(-2.66666666666666666667), lGuv[2][2], T(0)));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(1, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-1, +-1) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(2.0), lGp[0][2], T(0)));
    const T loep = fma(T(1.0), lGp[1][3], fma(T(-1.33333333333333333333), lGp[1][2], T(0)));
    const T leop = fma(T(0.666666666666666666667), lGp[2][2], fma(T(-1.0), lGp[2][1], T(0)));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(0.666666666666666666667), lGuv[1][2], T(0)));
    const T loeu = fma(T(1.0), lGuv[0][3], fma(T(-1.33333333333333333333), lGuv[0][2], T(0)));
    const T loou = fma(T(-0.666666666666666666667), lGuv[2][2], fma(T(1.0), lGuv[2][1], T(0)));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(1.33333333333333333333), lGuv[2][2], T(0)));
    const T leov = fma(T(0.666666666666666666667), lGuv[0][2], fma(T(-1.0), lGuv[0][1], T(0)));
    const T loov = fma(T(-0.666666666666666666667), lGuv[1][2], fma(T(1.0), lGuv[1][1], T(0)));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
  }
  {  // orbit (+-2, +-0) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(1.0), lGp[0][2], fma(T(1.0), lGp[0][1], fma(T(-0.5), lGp[0][0], T(0)))));
    const T loep = fma(T(1.0), lGp[1][3], fma(T(-0.666666666666666666667), lGp[1][2], fma(T(-1.0), lGp[1][1], fma(T(0.5), lGp[1][0], T(0)))));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(0.333333333333333333333), lGuv[1][2], fma(T(1.0), lGuv[1][1], fma(T(-0.5), lGuv[1][0], T(0)))));
    const T loeu = fma(T(1.0), lGuv[0][3], fma(T(-0.666666666666666666667), lGuv[0][2], fma(T(-1.0), lGuv[0][1], fma(T(0.5), lGuv[0][0], T(0)))));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(0.666666666666666666667), lGuv[2][2], T(0)));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(2, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-2, +-1) half cells
    const T leep = fma(T(0.666666666666666666667), lGp[0][3], fma(T(-0.5), lGp[0][2], T(0)));
    const T loep = fma(T(-0.5), lGp[1][3], fma(T(0.333333333333333333333), lGp[1][2], T(0)));
    const T leop = fma(T(-0.333333333333333333333), lGp[2][2], fma(T(0.25), lGp[2][1], T(0)));
    const T leeu = fma(T(0.333333333333333333333), lGuv[1][3], fma(T(-0.166666666666666666667), lGuv[1][2], T(0)));
    const T loeu = fma(T(-0.5), lGuv[0][3], fma(T(0.333333333333333333333), lGuv[0][2], T(0)));
    const T loou = fma(T(0.333333333333333333333), lGuv[2][2], fma(T(-0.25), lGuv[2][1], T(0)));
    const T leev = fma(T(0.333333333333333333333), lGuv[2][3], fma(T(-0.333333333333333333333), lGuv[2][2], T(0)));
    const T leov = fma(T(-0.333333333333333333333), lGuv[0][2], fma(T(0.25), lGuv[0][1], T(0)));
    const T loov = fma(T(0.333333333333333333333), lGuv[1][2], fma(T(-0.25), lGuv[1][1], T(0)));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.triple(1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
             T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov,
             c0p1[0], c0p1[1], c0p1[2]);
    S.triple(-1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
             T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov,
             c0m1[0], c0m1[1], c0m1[2]);
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

// family EH, transposed: lattice adjoints from output adjoints
template <typename T, typename Scatter>
__device__ __forceinline__ void af_sac_EH_adj(const Scatter& S, const T lGp[3][4], const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  {  // orbit (+-0, +-1) half cells
    const T leep = fma(T(2.66666666666666666667), lGp[0][3], fma(T(-4.0), lGp[0][2], fma(T(-2.0), lGp[0][1], fma(T(2.0), lGp[0][0], T(0)))));
    const T leop = fma(T(-2.0), lGp[2][3], fma(T(2.66666666666666666667), lGp[2][2], fma(T(2.0), lGp[2][1], fma(T(-2.0), lGp[2][0], T(0)))));
    const T leeu = fma(T(1.33333333333333333333), lGuv[1][3], fma(T(-2.66666666666666666667), lGuv[1][2], T(0)));
    const T leev = fma(T(1.33333333333333333333), lGuv[2][3], fma(T(-1.33333333333333333333), lGuv[2][2], fma(T(-2.0), lGuv[2][1], fma(T(2.0), lGuv[2][0], T(0)))));
    const T leov = fma(T(-2.0), lGuv[0][3], fma(T(2.66666666666666666667), lGuv[0][2], fma(T(2.0), lGuv[0][1], fma(T(-2.0), lGuv[0][0], T(0)))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S(0, 1, T(0) + leep + leop, T(0) + leeu, T(0) + leev + leov);
    S(0, -1, T(0) + leep - leop, T(0) + leeu, T(0) + leev - leov);
  }
  {  // orbit (+-0, +-2) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(1.0), lGp[0][2], fma(T(1.0), lGp[0][1], fma(T(-0.5), lGp[0][0], T(0)))));
    const T leop = fma(T(1.0), lGp[2][3], fma(T(-0.666666666666666666667), lGp[2][2], fma(T(-1.0), lGp[2][1], fma(T(0.5), lGp[2][0], T(0)))));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(0.666666666666666666667), lGuv[1][2], T(0)));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(0.333333333333333333333), lGuv[2][2], fma(T(1.0), lGuv[2][1], fma(T(-0.5), lGuv[2][0], T(0)))));
    const T leov = fma(T(1.0), lGuv[0][3], fma(T(-0.666666666666666666667), lGuv[0][2], fma(T(-1.0), lGuv[0][1], fma(T(0.5), lGuv[0][0], T(0)))));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S(0, 2, T(0) + leep + leop, T(0) + leeu, T(0) + leev + leov);
    S(0, -2, T(0) + leep - leop, T(0) + leeu, T(0) + leev - leov);
  }
  {  // orbit (+-1, +-0) half cells
    const T leep = fma(T(1.33333333333333333333), lGp[0][3], fma(T(-3.0), lGp[0][2], fma(T(2.0), lGp[0][1], T(0))));
    const T loep = fma(T(-0.666666666666666666667), lGp[1][2], fma(T(1.5), lGp[1][1], fma(T(-1.0), lGp[1][0], T(0))));
    const T leeu = fma(T(0.666666666666666666667), lGuv[1][3], fma(T(-2.0), lGuv[1][2], fma(T(2.0), lGuv[1][1], T(0))));
    const T loeu = fma(T(-0.666666666666666666667), lGuv[0][2], fma(T(1.5), lGuv[0][1], fma(T(-1.0), lGuv[0][0], T(0))));
    const T leev = fma(T(0.666666666666666666667), lGuv[2][3], fma(T(-1.0), lGuv[2][2], T(0)));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(1, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-1, +-1) half cells
    const T leep = fma(T(-1.33333333333333333333), lGp[0][3], fma(T(2.0), lGp[0][2], T(0)));
    const T loep = fma(T(0.666666666666666666667), lGp[1][2], fma(T(-1.0), lGp[1][1], T(0)));
    const T leop = fma(T(1.0), lGp[2][3], fma(T(-1.33333333333333333333), lGp[2][2], T(0)));
    const T leeu = fma(T(-0.666666666666666666667), lGuv[1][3], fma(T(1.33333333333333333333), lGuv[1][2], T(0)));
    const T loeu = fma(T(0.666666666666666666667), lGuv[0][2], fma(T(-1.0), lGuv[0][1], T(0)));
    const T loou = fma(T(-0.666666666666666666667), lGuv[2][2], fma(T(1.0), lGuv[2][1], T(0)));
    const T leev = fma(T(-0.666666666666666666667), lGuv[2][3], fma(T(0.666666666666666666667), lGuv[2][2], T(0)));
    const T leov = fma(T(1.0), lGuv[0][3], fma(T(-1.33333333333333333333), lGuv[0][2], T(0)));
    const T loov = fma(T(-0.666666666666666666667), lGuv[1][2], fma(T(1.0), lGuv[1][1], T(0)));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
  }
  {  // orbit (+-1, +-2) half cells
    const T leep = fma(T(0.666666666666666666667), lGp[0][3], fma(T(-0.5), lGp[0][2], T(0)));
    const T loep = fma(T(-0.333333333333333333333), lGp[1][2], fma(T(0.25), lGp[1][1], T(0)));
    const T leop = fma(T(-0.5), lGp[2][3], fma(T(0.333333333333333333333), lGp[2][2], T(0)));
    const T leeu = fma(T(0.333333333333333333333), lGuv[1][3], fma(T(-0.333333333333333333333), lGuv[1][2], T(0)));
    const T loeu = fma(T(-0.333333333333333333333), lGuv[0][2], fma(T(0.25), lGuv[0][1], T(0)));
    const T loou = fma(T(0.333333333333333333333), lGuv[2][2], fma(T(-0.25), lGuv[2][1], T(0)));
    const T leev = fma(T(0.333333333333333333333), lGuv[2][3], fma(T(-0.166666666666666666667), lGuv[2][2], T(0)));
    const T leov = fma(T(-0.5), lGuv[0][3], fma(T(0.333333333333333333333), lGuv[0][2], T(0)));
    const T loov = fma(T(0.333333333333333333333), lGuv[1][2], fma(T(-0.25), lGuv[1][1], T(0)));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 2, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -2, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
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

// family C, transposed: lattice adjoints from output adjoints
template <typename T, typename Scatter>
__device__ __forceinline__ void af_sac_C_adj(const Scatter& S, const T lGp[3][4], const T lGuv[3][4], T& lpK, T& luK, T& lvK) {
  {  // orbit (+-0, +-1) half cells
    const T leep = fma(T(-2.66666666666666666667), lGp[0][3], fma(T(2.0), lGp[0][1], T(0)));
    const T leop = fma(T(1.33333333333333333333), lGp[2][2], fma(T(-1.0), lGp[2][0], T(0)));
    const T leeu = fma(T(-1.33333333333333333333), lGuv[1][3], T(0));
    const T leev = fma(T(-1.33333333333333333333), lGuv[2][3], fma(T(2.0), lGuv[2][1], T(0)));
    const T leov = fma(T(1.33333333333333333333), lGuv[0][2], fma(T(-1.0), lGuv[0][0], T(0)));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S(0, 1, T(0) + leep + leop, T(0) + leeu, T(0) + leev + leov);
    S(0, -1, T(0) + leep - leop, T(0) + leeu, T(0) + leev - leov);
  }
  {  // orbit (+-1, +-0) half cells
    const T leep = fma(T(-2.66666666666666666667), lGp[0][3], fma(T(2.0), lGp[0][1], T(0)));
    const T loep = fma(T(1.33333333333333333333), lGp[1][2], fma(T(-1.0), lGp[1][0], T(0)));
    const T leeu = fma(T(-1.33333333333333333333), lGuv[1][3], fma(T(2.0), lGuv[1][1], T(0)));
    const T loeu = fma(T(1.33333333333333333333), lGuv[0][2], fma(T(-1.0), lGuv[0][0], T(0)));
    const T leev = fma(T(-1.33333333333333333333), lGuv[2][3], T(0));
    lpK -= T(2) * leep;
    luK -= T(2) * leeu;
    lvK -= T(2) * leev;
    S.pair(1, 0, T(0) + leep + loep, T(0) + leeu + loeu, T(0) + leev,
           T(0) + leep - loep, T(0) + leeu - loeu, T(0) + leev);
  }
  {  // orbit (+-1, +-1) half cells
    const T leep = fma(T(1.33333333333333333333), lGp[0][3], T(0));
    const T loep = fma(T(-0.666666666666666666667), lGp[1][2], T(0));
    const T leop = fma(T(-0.666666666666666666667), lGp[2][2], T(0));
    const T leeu = fma(T(0.666666666666666666667), lGuv[1][3], T(0));
    const T loeu = fma(T(-0.666666666666666666667), lGuv[0][2], T(0));
    const T loou = fma(T(0.5), lGuv[2][1], T(0));
    const T leev = fma(T(0.666666666666666666667), lGuv[2][3], T(0));
    const T leov = fma(T(-0.666666666666666666667), lGuv[0][2], T(0));
    const T loov = fma(T(0.5), lGuv[1][1], T(0));
    lpK -= T(4) * leep;
    luK -= T(4) * leeu;
    lvK -= T(4) * leev;
    S.pair(1, 1, T(0) + leep + loep + leop, T(0) + leeu + loeu + loou, T(0) + leev + leov + loov,
           T(0) + leep - loep + leop, T(0) + leeu - loeu - loou, T(0) + leev + leov - loov);
    S.pair(1, -1, T(0) + leep + loep - leop, T(0) + leeu + loeu - loou, T(0) + leev - leov - loov,
           T(0) + leep - loep - leop, T(0) + leeu - loeu + loou, T(0) + leev - leov + loov);
  }
}
