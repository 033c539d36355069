// kernels_d3q19.cu -- kernel instantiations for the D3Q19 lattice.
#include "kernels.cuh"

namespace lbm {

bool kernels_d3q19(int order, int coll, int fp32, KernelSet* ks)
{
    if (order == 4 && coll == 0) {
        *ks = fp32 ? make_set<kLatD3Q19, 4, 0, float>() : make_set<kLatD3Q19, 4, 0, double>();
        return true;
    }
    if (order == 4 && coll == 1) {
        *ks = fp32 ? make_set<kLatD3Q19, 4, 1, float>() : make_set<kLatD3Q19, 4, 1, double>();
        return true;
    }
    if (order == 6 && coll == 0) {
        *ks = fp32 ? make_set<kLatD3Q19, 6, 0, float>() : make_set<kLatD3Q19, 6, 0, double>();
        return true;
    }
    if (order == 6 && coll == 1) {
        *ks = fp32 ? make_set<kLatD3Q19, 6, 1, float>() : make_set<kLatD3Q19, 6, 1, double>();
        return true;
    }
    return false;
}

}  // namespace lbm
