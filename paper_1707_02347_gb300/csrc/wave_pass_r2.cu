// wave_pass_r2.cu -- instantiations of the pass kernel for stencil radius 2 (SO 4).
#include "wave_pass.cuh"

namespace wave {

bool launch_pass_r2(int T, const CUtensorMap& mapA, const CUtensorMap& mapP, const CUtensorMap& mapK,
                    const PassArgs& a, int threads, size_t smem, long long blocks, cudaStream_t st, cudaError_t* err)
{
    switch (T) {
        case 1: *err = detail::launch_impl<2, 1>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 2: *err = detail::launch_impl<2, 2>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 3: *err = detail::launch_impl<2, 3>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        case 4: *err = detail::launch_impl<2, 4>(mapA, mapP, mapK, a, threads, smem, blocks, st); return true;
        default: return false;
    }
}

int pass_max_threads_r2(int T)
{
    switch (T) {
        case 1: return detail::Cfg<2, 1>::MAXT;
        case 2: return detail::Cfg<2, 2>::MAXT;
        case 3: return detail::Cfg<2, 3>::MAXT;
        case 4: return detail::Cfg<2, 4>::MAXT;
        default: return 0;
    }
}

int pass_prefetch_r2(int T)
{
    switch (T) {
        case 1: return detail::Cfg<2, 1>::D;
        case 2: return detail::Cfg<2, 2>::D;
        case 3: return detail::Cfg<2, 3>::D;
        case 4: return detail::Cfg<2, 4>::D;
        default: return 0;
    }
}

}  // namespace wave
