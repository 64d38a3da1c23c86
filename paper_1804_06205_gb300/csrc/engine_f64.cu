// FP64 batch engine: the plain FP64 path, absolute FP64 positions and FP64
// arithmetic in every kernel.
#include "engine_impl.cuh"

namespace dpd {

BatchBase *make_batch_f64(const BatchConfig &bc, int *rc, std::string *err) {
    BatchEngine<PF64> *e = new BatchEngine<PF64>(bc);
    *rc = e->init();
    if (*rc) {
        *err = e->last_error();
        delete e;
        return nullptr;
    }
    return e;
}

}  // namespace dpd
