// FP32 batch engine: FP32 pair and bond forces, positions stored as FP32 offsets
// inside their cell; FP64 for the initial wrap, the cell keys and the reductions.
#include "engine_impl.cuh"

namespace dpd {

BatchBase *make_batch_f32(const BatchConfig &bc, int *rc, std::string *err) {
    BatchEngine<PF32> *e = new BatchEngine<PF32>(bc);
    *rc = e->init();
    if (*rc) {
        *err = e->last_error();
        delete e;
        return nullptr;
    }
    return e;
}

}  // namespace dpd
