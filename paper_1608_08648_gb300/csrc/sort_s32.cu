// The sort of 32-byte string keys (OS_S32): the method on word 0 with the
// original index as payload, refinement of tied runs by words 1-3, gather.
#include "strings.cuh"

namespace ossort {

int run_s32(RunArgs& a) {
    Ctx c;
    c.st = a.st;
    c.num_sms = a.num_sms;
    c.ar.base = static_cast<char*>(a.ws);
    c.ar.cap = a.ws_bytes;
    c.status = c.ar.take<uint32_t>(8);
    if (c.live()) os_memset_async(c.status, 0, 8 * sizeof(uint32_t), c.st);
    const uint32_t n = (uint32_t)a.n;
    const Str32* in = static_cast<const Str32*>(a.kin);
    Str32* out = static_cast<Str32*>(a.kout);
    uint64_t* P = c.ar.take<uint64_t>(n);
    uint32_t* I = c.ar.take<uint32_t>(n);
    uint64_t* Ps = c.ar.take<uint64_t>(n);
    uint32_t* Is = c.ar.take<uint32_t>(n);
    if (c.live() && n > 0)
        OS_LAUNCH(c.st, "k_str_init", k_str_init<<<grid_for(n, 256), 256, 0, c.st>>>(in, n, P, I));
    // The method on (word 0, original index).
    sort_top<KeyU64, true>(c, P, Ps, I, Is, n, a.prm, a.res);
    // Refinement buffers.
    const uint32_t nblk = (n + STR_BLK - 1) / STR_BLK;
    uint8_t* e[2] = {c.ar.take<uint8_t>(n), c.ar.take<uint8_t>(n)};
    uint32_t* blk = c.ar.take<uint32_t>(2 * (size_t)nblk + 2);
    uint32_t* tot = c.ar.take<uint32_t>(4);
    uint64_t* W = c.ar.take<uint64_t>(n);
    uint64_t* W2 = c.ar.take<uint64_t>(n);
    uint32_t* Iw = c.ar.take<uint32_t>(n);
    uint32_t* Iw2 = c.ar.take<uint32_t>(n);
    uint32_t* pos = c.ar.take<uint32_t>(n);
    uint32_t* seg = c.ar.take<uint32_t>((size_t)n / 2 + 2);
    const size_t sub_bytes = str_refine_bytes(n);
    char* sub = c.ar.take<char>(sub_bytes);
    // In place (in == out, as os_sort_host sorts): the gather goes through a copy.
    const bool in_place = a.kin == a.kout;
    Str32* tmp = c.ar.take<Str32>(in_place ? n : 0);
    uint32_t* vtmp = c.ar.take<uint32_t>(in_place && a.has_vals ? n : 0);
    a.res.str_keys = c.ar.take<Str32>(std::max<uint32_t>(a.prm.p, 2) - 1);
    a.res.str_map = a.prm.split == OS_DET ? a.res.det_index : nullptr;
    a.used = c.ar.used;
    a.status = c.status;
    if (!c.live()) return c.ar.failed ? OS_ERR_WS : OS_OK;
    if (n == 0) return OS_OK;
    const unsigned g = grid_for(n, 256);
    for (int w = 1; w < 4; ++w) {
        OS_LAUNCH(c.st, "k_str_eq",
                  k_str_eq<<<g, 256, 0, c.st>>>(w, in, Ps, Is, e[(w + 1) & 1], n, e[w & 1]));
        const uint8_t* ew = e[w & 1];
        OS_LAUNCH(c.st, "k_str_count", k_str_count<<<nblk, STR_NT, 0, c.st>>>(ew, n, blk));
        OS_LAUNCH(c.st, "k_str_scan", k_str_scan<<<1, 1024, 0, c.st>>>(blk, nblk, tot));
        OS_LAUNCH(c.st, "k_str_compact",
                  k_str_compact<<<nblk, STR_NT, 0, c.st>>>(w, in, Is, ew, n, blk, tot, W, Iw, pos, seg));
        uint32_t h_tot[2] = {0, 0};
        cudaError_t err = cudaMemcpyAsync(h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, c.st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(c.st);
        if (err != cudaSuccess) return OS_ERR_CUDA;
        if (h_tot[1] == 0) break;                       // no ties left
        Ctx sc = c;
        sc.ar = Arena{};
        sc.ar.base = sub;
        sc.ar.cap = sub_bytes;
        const SegSource src{nullptr, seg, h_tot[1], h_tot[0]};
        seg_core<KeyU64, true>(sc, src, bucket_classes<uint64_t>(), W, Iw, W2, Iw2, W, Iw,
                               sm_mix(a.prm.seed ^ (0x57A1ull + w)), nullptr);
        if (sc.ar.failed) return OS_ERR_WS;
        OS_LAUNCH(c.st, "k_str_put", k_str_put<<<grid_for(h_tot[0], 256), 256, 0, c.st>>>(Iw2, pos, tot, Is));
    }
    if (in_place) {
        OS_LAUNCH(c.st, "k_str_gather", k_str_gather<<<g, 256, 0, c.st>>>(in, a.vin, Is, n, tmp, vtmp));
        cudaError_t err = cudaMemcpyAsync(out, tmp, (size_t)n * sizeof(Str32), cudaMemcpyDeviceToDevice, c.st);
        if (err == cudaSuccess && a.has_vals)
            err = cudaMemcpyAsync(a.vout, vtmp, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c.st);
        if (err != cudaSuccess) return OS_ERR_CUDA;
    } else {
        OS_LAUNCH(c.st, "k_str_gather", k_str_gather<<<g, 256, 0, c.st>>>(in, a.vin, Is, n, out, a.vout));
    }
    if (a.res.p_used > 1)
        OS_LAUNCH(c.st, "k_str_splitters",
                  k_str_splitters<<<grid_for(a.res.p_used - 1, 256), 256, 0, c.st>>>(
                      in, a.res.spl_t, a.res.str_map, a.res.p_used - 1, static_cast<Str32*>(a.res.str_keys)));
    return OS_OK;
}

}  // namespace ossort
