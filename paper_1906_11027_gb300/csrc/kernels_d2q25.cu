// kernels_d2q25.cu -- kernel instantiations for the D2Q25 lattice.
#include "kernels.cuh"

namespace lbm {

bool kernels_d2q25(int order, int coll, int fp32, KernelSet* ks)
{
    if (order == 4 && coll == 0) {
        *ks = fp32 ? make_set<kLatD2Q25, 4, 0, float>() : make_set<kLatD2Q25, 4, 0, double>();
        return true;
    }
    if (order == 6 && coll == 0) {
        *ks = fp32 ? make_set<kLatD2Q25, 6, 0, float>() : make_set<kLatD2Q25, 6, 0, double>();
        return true;
    }
    if (order == 8 && coll == 0) {
        *ks = fp32 ? make_set<kLatD2Q25, 8, 0, float>() : make_set<kLatD2Q25, 8, 0, double>();
        return true;
    }
    if (order == 10 && coll == 0) {
        *ks = fp32 ? make_set<kLatD2Q25, 10, 0, float>() : make_set<kLatD2Q25, 10, 0, double>();
        return true;
    }
    if (order == 4 && coll == 2) {
        *ks = fp32 ? make_set<kLatD2Q25, 4, 2, float>() : make_set<kLatD2Q25, 4, 2, double>();
        return true;
    }
    if (order == 6 && coll == 2) {
        *ks = fp32 ? make_set<kLatD2Q25, 6, 2, float>() : make_set<kLatD2Q25, 6, 2, double>();
        return true;
    }
    if (order == 8 && coll == 2) {
        *ks = fp32 ? make_set<kLatD2Q25, 8, 2, float>() : make_set<kLatD2Q25, 8, 2, double>();
        return true;
    }
    if (order == 10 && coll == 2) {
        *ks = fp32 ? make_set<kLatD2Q25, 10, 2, float>() : make_set<kLatD2Q25, 10, 2, double>();
        return true;
    }
    return false;
}

}  // namespace lbm
