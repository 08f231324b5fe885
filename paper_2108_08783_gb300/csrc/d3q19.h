// D3Q19 velocity set of Sec. 2.1 in the library's canonical order, usable
// from host and device code:
//   0 rest; 1/2 +-x; 3/4 +-y; 5/6 +-z; 7/8 (+1,+1,0)/(-1,-1,0);
//   9/10 (+1,-1,0)/(-1,+1,0); 11/12 (+1,0,+1)/(-1,0,-1);
//   13/14 (+1,0,-1)/(-1,0,+1); 15/16 (0,+1,+1)/(0,-1,-1);
//   17/18 (0,+1,-1)/(0,-1,+1).
// Opposite directions are paired as (2p-1, 2p), p = 1..9.
#pragma once

#ifdef __CUDACC__
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

LBM_HD constexpr int dir_x(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
LBM_HD constexpr int dir_y(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
LBM_HD constexpr int dir_z(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
LBM_HD constexpr int dir_opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

}  // namespace lbm
