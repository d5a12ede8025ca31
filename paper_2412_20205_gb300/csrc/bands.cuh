// Band entries of the 1D factors as the kernels read them (internal).
#pragma once
#include "device.hpp"

namespace igamg {
namespace dev {

// x-direction band entry (row i, band b): the Toeplitz interior comes from the
// kernel parameters, the p boundary rows at each end from the band arrays.
template <typename T>
__device__ __forceinline__ T band_m(const LevelView<T>& L, int i, int b) {
    return (i >= L.tlo[0] && i < L.thi[0]) ? L.Mc[0][b] : L.Mb[0][b * L.m[0] + i];
}
template <typename T>
__device__ __forceinline__ T band_k(const LevelView<T>& L, int i, int b) {
    return (i >= L.tlo[0] && i < L.thi[0]) ? L.Kc[0][b] : L.Kb[0][b * L.m[0] + i];
}
// band entry of direction d (row i, band b) for d = 1, 2
template <typename T>
__device__ __forceinline__ T band_md(const LevelView<T>& L, int d, int i, int b) {
    return (i >= L.tlo[d] && i < L.thi[d]) ? L.Mc[d][b] : L.Mb[d][b * L.m[d] + i];
}
template <typename T>
__device__ __forceinline__ T band_kd(const LevelView<T>& L, int d, int i, int b) {
    return (i >= L.tlo[d] && i < L.thi[d]) ? L.Kc[d][b] : L.Kb[d][b * L.m[d] + i];
}

}  // namespace dev
}  // namespace igamg
