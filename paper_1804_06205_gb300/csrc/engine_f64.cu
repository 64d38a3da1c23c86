// FP64 engine: the plain FP64 path, absolute FP64 positions and FP64
// arithmetic in every kernel.
#include "engine_impl.cuh"

namespace dpd {

EngineBase *make_engine_f64(const Config &cfg, int *rc, std::string *err) {
    Engine<PF64> *e = new Engine<PF64>(cfg);
    *rc = e->init();
    if (*rc) {
        *err = e->last_error();
        delete e;
        return nullptr;
    }
    return e;
}

}  // namespace dpd
