// Checkpoint and resume of one flow: el_save_state / el_load_state.
//
// A coupled step (Algorithm 1) depends on the flow only through
//   - omega-hat (high and low parts), the AB2 history and N-hat of the
//     current level n (Sec. 3.1, Eqs. 8-10),
//   - the level pair holding level n (the fluid step of n reads level n from
//     it and writes the pair (n, n+1) the particle step blends, Sec. 3.2),
//     and the streamfunction pair when tracers use Eq. 11,
//   - every particle's split state (cell, offset, image, velocity), its
//     original index and reference position x(0),
// so the saved image holds exactly those, plus the step count.  Loading it
// into a flow created with the same descriptor and stepping on reproduces
// the uninterrupted run bit for bit (the re-binning cadence and block shape
// enter no result).
//
// Image layout (host byte order, every section a multiple of 8 bytes):
//   CkptHeader | omega-hat hi | lo | history | N-hat | level pair |
//   [streamfunction pair] | per non-empty species: cell, offset, [velocity],
//   image, id, x0 | FNV-1a 64-bit checksum of everything before it.
#include "common.cuh"

#include <cmath>
#include <cstring>
#include <vector>

using namespace el;

namespace {

constexpr char kMagic[8] = {'E', 'L', 'S', 'T', 'A', 'T', 'E', '1'};
constexpr uint32_t kVersion = 2;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    uint64_t total_bytes;       // the whole image, checksum included
    el_flow_desc desc;          // of the flow that saved it
    int64_t step;
    int64_t since_sort;
    int64_t np[EL_MAX_SPECIES];
    double st[EL_MAX_SPECIES];
    int32_t kinematic;          // 1: the prescribed field of Sec. 5.2 (parameters below)
    int32_t reserved;
    el_kinematic kin;
};

uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

size_t pad8(size_t x) { return (x + 7) & ~size_t(7); }

// One device range of the image (pointer, bytes).
struct Section {
    void* dev;
    size_t bytes;
};

std::vector<Section> sections(el_flow* f, const int64_t* np, const double* st, int64_t step) {
    std::vector<Section> s;
    const size_t nm = f->nmodes * sizeof(float2);
    s.push_back({f->what, nm});
    s.push_back({f->what_lo, nm});
    s.push_back({f->hist, nm});
    s.push_back({f->nhat_cur ? f->nhat_cur : f->nhat, nm});  // a batch FFT pool may hold it
    const int pair = (int)((step + 1) % 2);  // pair (n-1, n): level n in its second half
    s.push_back({f->snap[pair], f->n2 * sizeof(float4)});
    if (f->psi_plane >= 0) s.push_back({f->psi[pair], f->n2 * sizeof(float2)});
    for (int k = 0; k < f->d.max_species; k++) {
        if (np[k] <= 0) continue;
        const Species& sp = f->sp[k];
        const int c = sp.cur;
        const size_t m = (size_t)np[k];
        s.push_back({sp.cell[c], m * 4});
        s.push_back({sp.off[c], m * 8});
        if (st[k] > 0.0) s.push_back({sp.vel[c], m * 8});
        s.push_back({sp.img[c], m * 8});
        s.push_back({sp.id[c], m * 4});
        s.push_back({sp.x0, m * 16});
    }
    return s;
}

size_t image_bytes(const std::vector<Section>& s) {
    size_t b = pad8(sizeof(CkptHeader));
    for (const Section& x : s) b += pad8(x.bytes);
    return b + sizeof(uint64_t);
}

// Every per-particle section of the image, checked on the host before any of
// it reaches the device: a checksum proves the image intact, not valid, and
// the device path indexes memory with these values (the re-binning sort bins
// by cell, the readback scatters by id).  Cells must lie below n on both
// axes and ids must be a permutation of [0, np); offsets must lie in [0, 1)
// and velocities and x(0) be finite.  EL_CHECK_BOUNDS debug builds skip the
// offset range test (offsets index nothing: the gathers wrap their indices),
// so that their in-kernel invariant check can be exercised by an image.
const char* particle_sections_problem(const unsigned char* in, size_t at, int n, const int64_t* np,
                                      const double* st, int max_species) {
    std::vector<unsigned char> seen;
    for (int k = 0; k < max_species; k++) {
        if (np[k] <= 0) continue;
        const size_t m = (size_t)np[k];
        const unsigned char* cell = in + at;
        at += pad8(m * 4);
        const unsigned char* off = in + at;
        at += pad8(m * 8);
        const unsigned char* vel = nullptr;
        if (st[k] > 0.0) {
            vel = in + at;
            at += pad8(m * 8);
        }
        at += pad8(m * 8);  // image counts: any value is a valid periodic image
        const unsigned char* id = in + at;
        at += pad8(m * 4);
        const unsigned char* x0 = in + at;
        at += pad8(m * 16);
        seen.assign(m, 0);
        for (size_t p = 0; p < m; p++) {
            uint32_t c, q;
            float o[2], v[2];
            double x[2];
            std::memcpy(&c, cell + 4 * p, 4);
            if ((c & 0xffffu) >= (uint32_t)n || (c >> 16) >= (uint32_t)n) return "a cell index is not below n";
            std::memcpy(o, off + 8 * p, 8);
            if (!(std::isfinite(o[0]) && std::isfinite(o[1]))) return "an in-cell offset is not finite";
            if (!EL_CHECK_BOUNDS && !(o[0] >= 0.f && o[0] < 1.f && o[1] >= 0.f && o[1] < 1.f))
                return "an in-cell offset is outside [0, 1)";
            if (vel) {
                std::memcpy(v, vel + 8 * p, 8);
                if (!(std::isfinite(v[0]) && std::isfinite(v[1]))) return "a particle velocity is not finite";
            }
            std::memcpy(&q, id + 4 * p, 4);
            if (q >= m || seen[q]) return "the particle ids are not a permutation of [0, np)";
            seen[q] = 1;
            std::memcpy(x, x0 + 16 * p, 16);
            if (!(std::isfinite(x[0]) && std::isfinite(x[1]))) return "a reference position x(0) is not finite";
        }
    }
    return nullptr;
}

bool same_flow(const CkptHeader& h, const el_flow* f) {
    const el_flow_desc &a = h.desc, &b = f->d;
    return a.n == b.n && a.interp == b.interp && std::memcmp(&a.nu, &b.nu, sizeof(double)) == 0 &&
           std::memcmp(&a.dt, &b.dt, sizeof(double)) == 0 && a.ab2_mode == b.ab2_mode &&
           a.bspline_prefilter == b.bspline_prefilter && a.tracer_velocity == b.tracer_velocity &&
           h.kinematic == f->kinematic &&
           (!f->kinematic || std::memcmp(&h.kin, &f->kin, sizeof(el_kinematic)) == 0);
}

}  // namespace

extern "C" {

el_status el_save_state(el_flow* f, void* host_buf, size_t* bytes) {
    if (!f || !bytes) return EL_EINVAL;
    NvtxRange range("el_save_state");
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, sizeof kMagic);
    h.version = kVersion;
    h.header_bytes = (uint32_t)sizeof(CkptHeader);
    h.desc = f->d;
    h.step = f->step;
    h.since_sort = f->since_sort;
    h.kinematic = f->kinematic;
    h.kin = f->kin;
    for (int k = 0; k < f->d.max_species; k++) {
        h.np[k] = f->sp[k].np;
        h.st[k] = f->sp[k].st;
    }
    const std::vector<Section> secs = sections(f, h.np, h.st, h.step);
    const size_t need = image_bytes(secs);
    h.total_bytes = need;
    if (!host_buf) {
        *bytes = need;
        return EL_OK;
    }
    if (*bytes < need) {
        size_t have = *bytes;
        *bytes = need;
        return fail(f, EL_EINVAL, "buffer has %zu bytes, the state needs %zu", have, need);
    }
    unsigned char* out = static_cast<unsigned char*>(host_buf);
    std::memset(out, 0, need);
    std::memcpy(out, &h, sizeof h);
    size_t at = pad8(sizeof h);
    for (const Section& x : secs) {
        EL_CUDA_OK(f, cudaMemcpyAsync(out + at, x.dev, x.bytes, cudaMemcpyDeviceToHost, f->stream));
        at += pad8(x.bytes);
    }
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    const uint64_t sum = fnv1a(out, at);
    std::memcpy(out + at, &sum, sizeof sum);
    *bytes = need;
    return EL_OK;
}

el_status el_load_state(el_flow* f, const void* host_buf, size_t bytes) {
    if (!f || !host_buf) return EL_EINVAL;
    NvtxRange range("el_load_state");
    if (f->batch) return fail(f, EL_ESTATE, "flow belongs to a batch: remove it before loading");
    const unsigned char* in = static_cast<const unsigned char*>(host_buf);
    CkptHeader h{};
    if (bytes < sizeof h + sizeof(uint64_t)) return fail(f, EL_EINVAL, "state image too short");
    std::memcpy(&h, in, sizeof h);
    if (std::memcmp(h.magic, kMagic, sizeof kMagic) != 0) return fail(f, EL_EINVAL, "not a state image");
    if (h.version != kVersion || h.header_bytes != sizeof h)
        return fail(f, EL_EINVAL, "state image version %u not supported", h.version);
    if (h.total_bytes != bytes)
        return fail(f, EL_EINVAL, "state image is %zu bytes, its header says %llu", bytes,
                    (unsigned long long)h.total_bytes);
    uint64_t sum = 0;
    std::memcpy(&sum, in + bytes - sizeof sum, sizeof sum);
    if (fnv1a(in, bytes - sizeof sum) != sum) return fail(f, EL_EINVAL, "state image checksum mismatch");
    if (!same_flow(h, f))
        return fail(f, EL_EINVAL,
                    "state image was saved by a flow with another n, scheme, nu, dt, mode or field");
    if (h.step < 0 || h.since_sort < 0) return fail(f, EL_EINVAL, "state image has a negative step");
    for (int k = 0; k < EL_MAX_SPECIES; k++) {
        if (h.np[k] < 0 || (h.np[k] > 0 && k >= f->d.max_species))
            return fail(f, EL_EINVAL, "state image has particles in species %d this flow lacks", k);
        if (h.np[k] > f->d.max_particles)
            return fail(f, EL_EINVAL, "species %d has %lld particles, more than max_particles", k,
                        (long long)h.np[k]);
        if (h.np[k] > 0 && !(std::isfinite(h.st[k]) && h.st[k] >= 0.0))
            return fail(f, EL_EINVAL, "state image has a bad Stokes number");
    }
    // the image must hold exactly the sections its header declares (checked
    // before any of them is read), and every particle's state must be valid
    {
        const std::vector<Section> want = sections(f, h.np, h.st, h.step);  // sizes only
        if (image_bytes(want) != bytes)
            return fail(f, EL_EINVAL, "state image is %zu bytes, its particle counts need %zu", bytes,
                        image_bytes(want));
        size_t at = pad8(sizeof h);
        for (int q = 0; q < 5 + (f->psi_plane >= 0 ? 1 : 0); q++) at += pad8(want[q].bytes);
        if (const char* why = particle_sections_problem(in, at, f->n, h.np, h.st, f->d.max_species))
            return fail(f, EL_EINVAL, "state image refused: %s", why);
    }
    // room for every species, checked before anything changes
    if (!species_fit(f, h.np)) return fail(f, EL_EINVAL, "particle pool too small for the state image");
    for (int k = 0; k < f->d.max_species; k++)
        if (!carve_species_slot(f, k, h.np[k])) return fail(f, EL_EINVAL, "particle pool exhausted");
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    for (int k = 0; k < f->d.max_species; k++) {
        f->sp[k].np = h.np[k];
        f->sp[k].st = h.np[k] > 0 ? h.st[k] : 0.0;
        f->sp[k].cur = 0;
    }
    f->step = h.step;
    f->since_sort = h.since_sort;
    const std::vector<Section> secs = sections(f, h.np, h.st, h.step);
    size_t at = pad8(sizeof h);
    for (const Section& x : secs) {
        EL_CUDA_OK(f, cudaMemcpyAsync(x.dev, in + at, x.bytes, cudaMemcpyHostToDevice, f->stream));
        at += pad8(x.bytes);
    }
    for (int k = 0; k < f->d.max_species; k++) EL_TRY(particles_restore_table(f, k));
    EL_TRY(fluid_refresh_planes(f));
    drop_graphs(f);
    EL_CUDA_OK(f, cudaStreamSynchronize(f->stream));
    return EL_OK;
}

}  // extern "C"
