// FP32 engine: FP32 pair and bond forces, positions stored as FP32 offsets
// inside their cell, FP64 for the wrap, the cell keys and the reductions.
#include "engine_impl.cuh"

namespace dpd {

EngineBase *make_engine_f32(const Config &cfg, int *rc, std::string *err) {
    Engine<PF32> *e = new Engine<PF32>(cfg);
    *rc = e->init();
    if (*rc) {
        *err = e->last_error();
        delete e;
        return nullptr;
    }
    return e;
}

}  // namespace dpd
