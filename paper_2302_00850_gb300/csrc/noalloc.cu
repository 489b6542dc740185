// cola_mdagm_apply_noalloc: the normal operator M^dag M without any device
// allocation, for callers that cannot allocate device memory at the time of
// the call.
//
// Typical such callers: code that runs where a device allocation would
// implicitly synchronise the GPU or must not fail (a fixed-memory service, a
// callback), or a host program that reserves all device memory up front.  cola_mdagm_apply allocates its two
// temporaries in the gauge handle on first use; this variant instead uses
// one file-scope device array of fixed size, kStaticScratchBytes (64 MiB),
// that lives in the library's device image.  A GPU that has loaded this part
// of the library keeps that array until the process exits.  With lazy module
// loading (the CUDA default) that happens at the first call on the device;
// with CUDA_MODULE_LOADING=EAGER every process that loads libcola reserves it
// on every device it uses, whether or not it ever calls this entry point.
//
// The scratch holds one packed spinor field per right-hand side in the
// requested precision: the even-odd operator puts its odd-parity temporary
// H_oe in and its even-parity temporary Mhat in into the two disjoint
// parity halves of that field, and the whole-lattice operator uses it for
// D in.  So a call needs cola_spinor_bytes(lat, prec, nrhs) bytes of scratch
// and is rejected (COLA_ERR_ARG) above 64 MiB: e.g. FP64 up to V = 349,525
// sites for one right-hand side, FP32 up to 699,050, FP16 up to 1,290,555.
//
// Every call shares the one array and leaves its last contents behind.  Each
// temporary is written in full before it is read, so nothing has to start at
// zero; but calls whose work overlaps on the GPU (on different streams, or
// from several threads without ordering) race on the array.
#include "cola_impl.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch in the current device's context.  In
// host code the symbol name is only a host-side handle, never a device
// address.  The lookup is repeated on every call rather than cached: after a
// cudaDeviceReset, or when the primary context is released and created again,
// the library's device code is loaded anew and the array can sit at another
// address, so a cached pointer would be stale.  Once the device code is
// loaded in the current context the lookup is a host-side table query; the
// first call in a context may load that code.
cola_status static_scratch(void **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cola::cuda_check(e, "cudaGetSymbolAddress(static scratch)");
    *out = p;
    return COLA_OK;
}

cola_status arg_error(const char *msg) {
    cola::set_error(msg);
    return COLA_ERR_ARG;
}

}  // namespace

extern "C" cola_status cola_mdagm_apply_noalloc(cola_gauge g, void *out, const void *in, int op, cola_prec prec,
                                                int nrhs, cudaStream_t stream) {
    if (!g || !out || !in) return arg_error("null argument to cola_mdagm_apply_noalloc");
    if (op != COLA_OP_FULL && op != COLA_OP_EO) return arg_error("op must be COLA_OP_FULL or COLA_OP_EO");
    if (out == in) return arg_error("out must not alias in");
    if (prec < 0 || prec > 2) return arg_error("precision must be COLA_F64, COLA_F32 or COLA_F16");
    if (!g->links[prec]) {
        cola::set_error("gauge handle holds no links of this precision");
        return COLA_ERR_UNSUPPORTED;
    }
    if (nrhs < 1 || nrhs > 65535) return arg_error("nrhs must be in 1..65535");
    const size_t need = 2 * cola::spinor_parity_bytes(prec, g->geom.Vh) * (size_t)nrhs;
    if (need > kStaticScratchBytes) {
        cola::set_error("cola_mdagm_apply_noalloc needs " + std::to_string(need) +
                        " bytes of scratch; its static scratch holds " + std::to_string(kStaticScratchBytes) +
                        " bytes (64 MiB): use cola_mdagm_apply for this size");
        return COLA_ERR_ARG;
    }
    void *w = nullptr;
    cola_status st = static_scratch(&w);
    if (st != COLA_OK) return st;
    // t (odd half) and mp (even half) share the one scratch field
    return cola::apply_mdagm(g, prec, op, out, in, w, w, nrhs, nullptr, false, stream);
}
