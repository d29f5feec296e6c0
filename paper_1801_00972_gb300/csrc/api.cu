// Host side of libpic: argument checks, device allocation, the step driver and
// the query calls of the C ABI declared in include/pic.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "pic_internal.cuh"

namespace pic {

void* dev_alloc(pic_ctx* c, size_t bytes)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes < 16 ? 16 : bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->allocs.push_back(p);
    return p;
}

cudaEvent_t prof_begin(pic_ctx* c)
{
    if (!c->prof) return nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, c->stream);
    return e;
}

void prof_end(pic_ctx* c, cudaEvent_t start, bool push)
{
    if (!c->prof || !start) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, c->stream);
    (push ? c->ev_push : c->ev_solve).emplace_back(start, e);
}

int grid_for(int64_t n, int threads, int max_blocks)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}

}  // namespace pic

using namespace pic;

namespace {

thread_local std::string g_init_error;

pic_status fail(pic_ctx* c, pic_status s, const std::string& msg)
{
    if (c) c->err = msg;
    else g_init_error = msg;
    return s;
}

pic_status cuda_fail(pic_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, PIC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// zero every moment window (rf average, phase bins, fine grid) on `st`
// (synchronous memsets when st is null)
cudaError_t clear_moments(pic_ctx* c, cudaStream_t st)
{
    const size_t nb = (size_t)c->nph;
    const size_t sz[10] = {sizeof(double) * 4 * c->nodes * nb, sizeof(double) * 4 * c->nodes * nb,
                           sizeof(double) * c->nodes * nb, sizeof(unsigned long long) * nb,
                           sizeof(double) * 4 * c->nfine, sizeof(double) * 4 * c->nfine,
                           sizeof(double) * c->nodes * nb, sizeof(double) * c->nodes * nb,
                           sizeof(float) * 5 * c->nodes, sizeof(float) * 5 * c->nodes};
    void* p[10] = {c->mom[0], c->mom[1], c->mphi, c->d_bsteps, c->fine[0], c->fine[1], c->mke[0], c->mke[1],
                   c->mom32[0], c->mom32[1]};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 10 && e == cudaSuccess; ++q)
        if (p[q]) e = st ? cudaMemsetAsync(p[q], 0, sz[q], st) : cudaMemset(p[q], 0, sz[q]);
    return e;
}

// one moment sample after the step's solve: the phase bin, node moments and phi, fine grid
void launch_moments_all(pic_ctx* c)
{
    if (c->nph > 1) launch_phase_bin(c);
    if (c->prec == PIC_MIXED) launch_moments32(c);
    else launch_moments64(c);
    launch_moments_phi(c);
    if (c->nfine) launch_fine(c);
}

// averages of phase bins [b0, b1) over `steps` samples into out (layout of pic_moments)
pic_status moments_window(pic_ctx* c, int what, int b0, int b1, int64_t steps, double* out)
{
    if (what >= 5) {
        // temperature (eV) of the window's node-weighted velocities: (m / 3e) (<v^2> - |<v>|^2)
        const int sp = what - 5;
        const size_t N = c->nodes, nb = (size_t)(b1 - b0);
        std::vector<double> m(4 * N * nb), k(N * nb);
        cudaError_t e = cudaMemcpy(m.data(), c->mom[sp] + 4 * N * (size_t)b0, sizeof(double) * m.size(),
                                   cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(k.data(), c->mke[sp] + N * (size_t)b0, sizeof(double) * k.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "moments copy");
        const double m3e = (2.0 / 3.0) * c->hm[sp];
        for (size_t q = 0; q < N; ++q) {
            double s[5] = {0, 0, 0, 0, 0};
            for (size_t b = 0; b < nb; ++b) {
                for (int a = 0; a < 4; ++a) s[a] += m[4 * (b * N + q) + a];
                s[4] += k[b * N + q];
            }
            if (!(s[0] > 0.0)) { out[q] = 0.0; continue; }
            const double u0 = s[1] / s[0], u1 = s[2] / s[0], u2 = s[3] / s[0];
            out[q] = m3e * (s[4] / s[0] - ((u0 * u0 + u1 * u1) + u2 * u2));
        }
        return PIC_OK;
    }
    const size_t N = c->nodes, len = (what >= 3 ? 3 : 1) * N, w = what == 0 ? 1 : 4;
    std::vector<double> m(w * N * (size_t)(b1 - b0));
    const double* src = what == 0 ? c->mphi : c->mom[(what - 1) % 2];
    const cudaError_t e = cudaMemcpy(m.data(), src + w * N * (size_t)b0, sizeof(double) * m.size(),
                                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments copy");
    for (size_t q = 0; q < len; ++q) out[q] = 0.0;
    for (int b = 0; b < b1 - b0; ++b) {
        const double* mb = m.data() + w * N * (size_t)b;
        for (size_t q = 0; q < N; ++q) {
            if (what == 0) out[q] += mb[q];
            else if (what <= 2) out[q] += mb[4 * q];
            else
                for (int a = 0; a < 3; ++a) out[3 * q + a] += mb[4 * q + 1 + a];
        }
    }
    const double scale = what == 0 ? 1.0 / (double)steps : c->W / ((c->dx * c->dx * c->dx) * (double)steps);
    for (size_t q = 0; q < len; ++q) out[q] *= scale;
    return PIC_OK;
}

// cell index and in-cell fraction along one axis, clamped into the mesh
inline void locate1(double x, double dx, int n, int& i, double& f)
{
    const double q = x / dx;
    i = (int)std::floor(q);
    if (i > n - 1) i = n - 1;
    if (i < 0) i = 0;
    f = q - (double)i;
}

double v_bottom(const pic_ctx* c)
{
    const double t = (double)c->step * c->dt;
    return c->el.v_dc + c->el.v_rf * std::sin((2.0 * kPI * c->el.f_rf) * t + c->el.phase);
}

double rho_scale(const pic_ctx* c)
{
    const double dx = c->dx;
    return (((kQE * c->W) / (dx * dx * dx)) * 0x1p-42) / kEPS0;
}

// device error word and pending solve status
pic_status check(pic_ctx* c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    int err = 0;
    e = cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error word");
    if (err == PIC_ECAPACITY) return fail(c, PIC_ECAPACITY, "particle or ionization-product capacity exceeded");
    if (err == PIC_ENONFINITE)
        return fail(c, PIC_ENONFINITE, "non-finite particle state or a particle moved more than one box length");
    if (err != 0) return fail(c, PIC_ECUDA, "device error " + std::to_string(err));
    int sf = 0;
    e = cudaMemcpy(&sf, c->d_solve_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "solve flag");
    if (sf != 0) {
        cudaMemset(c->d_solve_flag, 0, sizeof(int));
        if (sf == PIC_ENONFINITE) return fail(c, PIC_ENONFINITE, "Poisson solve: non-finite residual");
        return fail(c, PIC_ENOTCONV, "Poisson solve did not reach the tolerance within max_cycles");
    }
    return PIC_OK;
}

void deposit_particles(pic_ctx* c)
{
    if (c->prec == PIC_MIXED) launch_deposit32(c);
    else launch_deposit64(c);
}

pic_status solve_now(pic_ctx* c, double tol, int* iters, double* res)
{
    cudaEvent_t ev = prof_begin(c);
    launch_rhs(c, rho_scale(c), v_bottom(c), c->el.v_top, true);
    int it = 0;
    const pic_status s = mg_solve(c, v_bottom(c), c->el.v_top, tol, c->max_cycles, &it, res);
    prof_end(c, ev, false);
    if (c->prof) c->prof_iters += it;
    if (iters) *iters = it;
    return s;
}

void drop_events(pic_ctx* c)
{
    for (auto* v : {&c->ev_push, &c->ev_solve}) {
        for (auto& pr : *v) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        v->clear();
    }
    c->prof_iters = 0;
}

void drop_events(pic_ctx* c);

void destroy(pic_ctx* c)
{
    if (!c) return;
    drop_events(c);
    for (cudaGraphExec_t g : {c->g_pre, c->g_push[0], c->g_push[1], c->g_solve, c->g_post[0][0], c->g_post[0][1],
                              c->g_post[1][0], c->g_post[1][1], c->g_mom[0], c->g_mom[1]})
        if (g) cudaGraphExecDestroy(g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->aux2) cudaStreamDestroy(c->aux2);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    for (void* p : c->allocs) cudaFree(p);
    delete c;
}

bool finite_all(const double* p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

namespace pic {
void set_global_error(const char* msg) { g_init_error = msg; }
}  // namespace pic

extern "C" {

const char* pic_last_error(const pic_ctx* ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

void pic_destroy(pic_ctx* ctx)
{
    if (ctx) cudaStreamSynchronize(ctx->stream);
    destroy(ctx);
}

int64_t pic_step_index(const pic_ctx* ctx) { return ctx ? ctx->step : -1; }

}  // extern "C"

namespace {

// pic_init and pic_init_plasma: t_ev == nullptr takes the particles from the
// host arrays of `run`, else draws run->n[sp] particles of species sp at
// temperature t_ev[sp] on the device
pic_status init_run(const pic_mesh* mesh, const pic_electrodes* el, const pic_gas* gas, const pic_grains* grains,
                    const pic_run* run, const double* t_ev, void* cuda_stream, pic_ctx** out)
{
    g_init_error.clear();
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh || !el || !gas || !grains || !run) return fail(nullptr, PIC_EINVAL, "NULL argument");
    const int nx = mesh->nx, ny = mesh->ny, nz = mesh->nz;
    if (nx < 4 || ny < 4 || nz < 2 || nx % 2 || ny % 2)
        return fail(nullptr, PIC_EINVAL, "mesh: nx, ny must be even and >= 4, nz >= 2");
    if ((double)nx * ny * (nz + 1) > 2.0e9) return fail(nullptr, PIC_EINVAL, "mesh too large");
    if (!(mesh->dx > 0.0) || !std::isfinite(mesh->dx)) return fail(nullptr, PIC_EINVAL, "mesh: dx must be > 0");
    const double elv[5] = {el->v_dc, el->v_rf, el->f_rf, el->phase, el->v_top};
    if (!finite_all(elv, 5)) return fail(nullptr, PIC_EINVAL, "electrodes: non-finite value");
    if (gas->n_xs < 2 || !gas->xs_host || !(gas->de_e > 0) || !(gas->de_i > 0) || !(gas->n_gas >= 0) ||
        !(gas->t_gas >= 0) || !(gas->nu_max_e >= 0) || !(gas->nu_max_i >= 0))
        return fail(nullptr, PIC_EINVAL, "gas: need n_xs >= 2, tables, de > 0, non-negative densities and bounds");
    if (!finite_all(gas->xs_host, 5 * (size_t)gas->n_xs)) return fail(nullptr, PIC_EINVAL, "gas: non-finite table");
    if (grains->n < 0 || (grains->n > 0 && (!grains->pos_host || !grains->radius_host)))
        return fail(nullptr, PIC_EINVAL, "grains: bad count or NULL arrays");
    if (!(run->dt > 0.0) || !(run->weight >= 0.0) || run->md_sub < 1 || run->sort_every < 0 ||
        (run->prec != PIC_FP64 && run->prec != PIC_MIXED) || !(run->tol > 0.0) || run->max_cycles < 1)
        return fail(nullptr, PIC_EINVAL, "run: need dt > 0, weight >= 0, md_sub >= 1, sort_every >= 0, prec 0/1, "
                                         "tol > 0, max_cycles >= 1");
    if (run->eepf_bins < 0 || run->eepf_bins > 65536 || (run->eepf_bins > 0 && !(run->eepf_de_ev > 0.0)))
        return fail(nullptr, PIC_EINVAL, "run: eepf_bins in [0, 65536] and eepf_de_ev > 0 when bins > 0");
    {
        const bool any = run->fine_n[0] != 0 || run->fine_n[1] != 0 || run->fine_n[2] != 0;
        bool fine_ok = true;
        for (int a = 0; a < 3; ++a)
            fine_ok = fine_ok && (any ? run->fine_n[a] >= 1 && run->fine_n[a] <= 1024 : true);
        if (any)
            fine_ok = fine_ok && run->fine_h > 0.0 && std::isfinite(run->fine_h) && finite_all(run->fine_origin, 3);
        if (run->mom_phases < 0 || run->mom_phases > 1024 || !fine_ok ||
            ((run->mom_phases > 1 || any) && !(run->flags & PIC_F_MOMENTS)))
            return fail(nullptr, PIC_EINVAL, "run: mom_phases in [0, 1024]; fine_n all 0 or all in [1, 1024] with "
                                             "fine_h > 0 and a finite origin; both need PIC_F_MOMENTS");
    }
    if ((run->flags & PIC_F_COULOMB) && !(run->coulomb_log > 0.0 && run->coulomb_log < 1e3))
        return fail(nullptr, PIC_EINVAL, "run: PIC_F_COULOMB needs a Coulomb logarithm in (0, 1000)");
    if (run->prec == PIC_MIXED && (nx > 1024 || ny > 1024 || nz > 2047))
        return fail(nullptr, PIC_EINVAL, "mesh: mixed precision packs the cell as i | j << 10 | k << 20, so nx, ny "
                                         "<= 1024 and nz <= 2047");
    const double Lx = nx * mesh->dx, Ly = ny * mesh->dx, Lz = nz * mesh->dx;
    for (int sp = 0; sp < 2; ++sp) {
        if (run->n[sp] < 0 || run->capacity[sp] < run->n[sp] || run->capacity[sp] > 0x7fffffffLL)
            return fail(nullptr, PIC_EINVAL, "run: need 0 <= n <= capacity < 2^31");
        if (t_ev) {
            if (!(t_ev[sp] >= 0.0) || !std::isfinite(t_ev[sp]))
                return fail(nullptr, PIC_EINVAL, "plasma: temperatures must be finite and >= 0");
            continue;
        }
        if (run->n[sp] > 0 && (!run->x_host[sp] || !run->v_host[sp] || !run->id_host[sp]))
            return fail(nullptr, PIC_EINVAL, "run: NULL particle arrays");
        // each particle is checked (finite, inside the box) where it is converted, on the device
    }
    if (t_ev && run->n[0] + run->n[1] > 0xFFFFFFFFLL)
        return fail(nullptr, PIC_EINVAL, "plasma: n_e + n_i must fit the 32-bit particle ids");
    // grains: inside the box, one cell clear of both electrodes, <= 8 per MD cell
    std::vector<int> gcell(3 * (size_t)grains->n);
    for (int g = 0; g < grains->n; ++g) {
        const double* p = grains->pos_host + 3 * g;
        if (!finite_all(p, 3) || p[0] < 0 || p[0] >= Lx || p[1] < 0 || p[1] >= Ly || p[2] < 0 || p[2] >= Lz ||
            !(grains->radius_host[g] > 0.0) || !(grains->radius_host[g] < mesh->dx))
            return fail(nullptr, PIC_EINVAL, "grains: centre outside the box or radius not in (0, dx)");
        double f;
        locate1(p[0], mesh->dx, nx, gcell[3 * g], f);
        locate1(p[1], mesh->dx, ny, gcell[3 * g + 1], f);
        locate1(p[2], mesh->dx, nz, gcell[3 * g + 2], f);
        gcell[3 * g] = (int)std::floor(p[0] / mesh->dx);
        gcell[3 * g + 1] = (int)std::floor(p[1] / mesh->dx);
        gcell[3 * g + 2] = (int)std::floor(p[2] / mesh->dx);
        if (gcell[3 * g + 2] < 1 || gcell[3 * g + 2] > nz - 2)
            return fail(nullptr, PIC_EINVAL, "grains: a grain's cell must be at least one cell from each electrode");
        if (t_ev && !(1.5 * grains->radius_host[g] < mesh->dx))
            return fail(nullptr, PIC_EINVAL, "plasma: the sampler keeps 1.5 grain radii clear, so radii must be "
                                             "below dx / 1.5");
    }
    const size_t cells = (size_t)nx * ny * nz, nodes = (size_t)nx * ny * (nz + 1);
    std::vector<int> cell_ng(cells, 0), cell_g(cells * kMaxG, 0);
    for (int g = 0; g < grains->n; ++g)
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const int i = (gcell[3 * g] + di + nx) % nx, j = (gcell[3 * g + 1] + dj + ny) % ny,
                              k = gcell[3 * g + 2] + dk;
                    const size_t ci = ((size_t)k * ny + j) * nx + i;
                    if (cell_ng[ci] >= kMaxG) return fail(nullptr, PIC_EINVAL, "grains: more than 8 per MD cell");
                    cell_g[ci * kMaxG + cell_ng[ci]++] = g;
                }

    pic_ctx* c = new (std::nothrow) pic_ctx();
    if (!c) return fail(nullptr, PIC_ENOMEM, "host allocation");
    c->nx = nx; c->ny = ny; c->nz = nz; c->dx = mesh->dx;
    c->Lx = Lx; c->Ly = Ly; c->Lz = Lz;
    c->nodes = nodes; c->cells = cells;
    c->el = *el;
    c->n_gas = gas->n_gas; c->t_gas = gas->t_gas; c->eps_exc = gas->eps_exc; c->eps_ion = gas->eps_ion;
    c->nu_max[0] = gas->nu_max_e; c->nu_max[1] = gas->nu_max_i; c->de[0] = gas->de_e; c->de[1] = gas->de_i;
    c->n_xs = gas->n_xs;
    c->ng = grains->n;
    c->prec = run->prec; c->flags = run->flags; c->md_sub = run->md_sub; c->sort_every = run->sort_every;
    c->coul_log = run->coulomb_log;
    c->eepf_bins = run->eepf_bins;
    c->eepf_de = run->eepf_de_ev;
    c->nph = run->mom_phases > 1 ? run->mom_phases : 1;
    c->f_rf = el->f_rf;
    c->rf_phase = el->phase;
    if (run->fine_n[0] > 0) {
        for (int a = 0; a < 3; ++a) { c->fine_n[a] = run->fine_n[a]; c->fine_o[a] = run->fine_origin[a]; }
        c->fine_h = run->fine_h;
        c->nfine = (size_t)run->fine_n[0] * (size_t)run->fine_n[1] * (size_t)run->fine_n[2];
    }
    c->max_cycles = run->max_cycles;
    c->W = run->weight; c->dt = run->dt; c->tol = run->tol;
    c->seed = run->seed; c->run_id = run->run_id;
    c->key = make_uint2((uint32_t)run->seed ^ run->run_id, (uint32_t)(run->seed >> 32));
    c->qm[0] = -kQE / kME; c->qm[1] = kQE / kMAR;
    c->hm[0] = (0.5 * kME) / kQE; c->hm[1] = (0.5 * kMAR) / kQE;
    c->pnull[0] = 1.0 - std::exp(-gas->nu_max_e * run->dt);
    c->pnull[1] = 1.0 - std::exp(-gas->nu_max_i * run->dt);
    c->sig_n = std::sqrt(kKB * gas->t_gas / kMAR);
    c->stream = (cudaStream_t)cuda_stream;
    c->step = 0;
    for (int sp = 0; sp < 2; ++sp) c->cap[sp] = std::max<int64_t>(run->capacity[sp], 1);
    c->child_cap = std::max<int64_t>(4096, std::max(c->cap[0], c->cap[1]) / 64);
    c->sp.scale = rho_scale(c);
    c->sp.inv_h2 = 1.0 / (mesh->dx * mesh->dx);
    c->sp.v_dc = el->v_dc; c->sp.v_rf = el->v_rf; c->sp.f_rf = el->f_rf; c->sp.phase = el->phase;
    c->sp.v_top = el->v_top; c->sp.dt = run->dt;

    const bool mixed = c->prec == PIC_MIXED;
    const size_t psz = mixed ? sizeof(float4) : sizeof(double4);
    bool ok = true;
    for (int sp = 0; sp < 2; ++sp) {
        c->pos[sp] = dev_alloc(c, psz * c->cap[sp]);
        c->vel[sp] = dev_alloc(c, psz * c->cap[sp]);
        c->pos_alt[sp] = dev_alloc(c, psz * c->cap[sp]);
        c->vel_alt[sp] = dev_alloc(c, psz * c->cap[sp]);
        ok = ok && c->pos[sp] && c->vel[sp] && c->pos_alt[sp] && c->vel_alt[sp];
    }
    c->d_nslot = (unsigned long long*)dev_alloc(c, 2 * sizeof(unsigned long long));
    c->d_cnt = (unsigned long long*)dev_alloc(c, PIC_C_N * sizeof(unsigned long long));
    c->d_live = (unsigned long long*)dev_alloc(c, 2 * sizeof(unsigned long long));
    c->d_err = (int*)dev_alloc(c, sizeof(int));
    c->d_nch = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long));
    c->d_next_id = (unsigned int*)dev_alloc(c, sizeof(unsigned int));
    c->d_child = (ChildRec*)dev_alloc(c, sizeof(ChildRec) * c->child_cap);
    if (mixed) {
        c->md_rescap = std::max<int64_t>(65536, std::max(c->cap[0], c->cap[1]) / 8);
        for (int sp = 0; sp < 2; ++sp) {
            c->md_res[sp] = (float4*)dev_alloc(c, sizeof(float4) * 2 * c->md_rescap);
            ok = ok && c->md_res[sp];
            c->md_list[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * c->cap[sp]);
            c->md_next[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * c->cap[sp]);
            c->mcc_list[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * c->cap[sp]);
            ok = ok && c->md_list[sp] && c->md_next[sp] && c->mcc_list[sp];
        }
        c->d_lists = (unsigned int*)dev_alloc(c, 6 * sizeof(unsigned int));
        ok = ok && c->d_lists && cudaMemset(c->d_lists, 0, 6 * sizeof(unsigned int)) == cudaSuccess;
    }
    c->rq = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * nodes);
    c->phi = (double*)dev_alloc(c, sizeof(double) * nodes);
    c->phi_alt = (double*)dev_alloc(c, sizeof(double) * nodes);
    c->f64 = (double*)dev_alloc(c, sizeof(double) * nodes);
    if (mixed) c->e32 = (float4*)dev_alloc(c, sizeof(float4) * nodes);
    else c->e64 = (double*)dev_alloc(c, sizeof(double) * 3 * nodes);
    c->d_norm = (double*)dev_alloc(c, 4 * sizeof(double));
    c->d_step = (uint32_t*)dev_alloc(c, sizeof(uint32_t));
    c->d_iters = (unsigned int*)dev_alloc(c, sizeof(unsigned int));
    c->d_res = (double*)dev_alloc(c, sizeof(double));
    c->d_solve_flag = (int*)dev_alloc(c, sizeof(int));
    c->d_iter_total = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long));
    c->d_vb_last = (double*)dev_alloc(c, sizeof(double));
    c->xs64 = (double*)dev_alloc(c, sizeof(double) * 5 * c->n_xs);
    c->xs32 = (float*)dev_alloc(c, sizeof(float) * 5 * c->n_xs);
    const int ng1 = std::max(c->ng, 1);
    c->gpos = (double*)dev_alloc(c, sizeof(double) * 3 * ng1);
    c->grad = (double*)dev_alloc(c, sizeof(double) * ng1);
    c->gcell = (int*)dev_alloc(c, sizeof(int) * 3 * ng1);
    c->gq = (double*)dev_alloc(c, sizeof(double) * ng1);
    c->gabs = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * 2 * ng1);
    c->gtab = (double*)dev_alloc(c, sizeof(double) * kTab * ng1);
    c->gtab32 = (float*)dev_alloc(c, sizeof(float) * kTab * ng1);
    c->gq32 = (float*)dev_alloc(c, sizeof(float) * ng1);
    c->goff32 = (float*)dev_alloc(c, sizeof(float) * 3 * ng1);
    c->gr2_32 = (float*)dev_alloc(c, sizeof(float) * ng1);
    c->cell_ng = (int*)dev_alloc(c, sizeof(int) * cells);
    c->cell_g = (int*)dev_alloc(c, sizeof(int) * cells * kMaxG);
    // sort keys: the mixed path sorts by tiles of up to 8 x 8 x 8 cells (the push's
    // unit of work), the FP64 path by cell
    for (int a = 0; a < 3; ++a) {
        const int n = a == 0 ? nx : a == 1 ? ny : nz;
        c->tile[a] = mixed ? std::min(8, n) : 1;
        c->ntile[a] = (n + c->tile[a] - 1) / c->tile[a];
    }
    c->ntiles = (int64_t)c->ntile[0] * c->ntile[1] * c->ntile[2];
    c->nkeys = mixed ? (size_t)c->ntiles * (size_t)(c->tile[0] * c->tile[1] * c->tile[2]) : cells;
    c->cursor = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (c->nkeys + 1));
    c->nkeys_cap = c->nkeys;
    c->ntiles_cap = c->ntiles;
    if (mixed)
        for (int sp = 0; sp < 2; ++sp) {
            c->tstart[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (size_t)(c->ntiles + 1));
            ok = ok && c->tstart[sp];
        }
    if (c->flags & PIC_F_COULOMB)
        for (int sp = 0; sp < 2; ++sp) {
            c->cs_end[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (cells + 1));
            c->cs_idx[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (size_t)std::max<int64_t>(c->cap[sp], 1));
            c->cs_key[sp] =
                (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * (size_t)std::max<int64_t>(c->cap[sp], 1));
            c->cs_cell[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (size_t)std::max<int64_t>(c->cap[sp], 1));
            c->cs_ord[sp] = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (size_t)std::max<int64_t>(c->cap[sp], 1));
            ok = ok && c->cs_end[sp] && c->cs_idx[sp] && c->cs_key[sp] && c->cs_cell[sp] && c->cs_ord[sp];
        }
    if (c->eepf_bins > 0) {
        c->eepf = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * (size_t)nz * (c->eepf_bins + 1));
        ok = ok && c->eepf;
        if (c->eepf) cudaMemset(c->eepf, 0, sizeof(unsigned long long) * (size_t)nz * (c->eepf_bins + 1));
    }
    if (c->flags & PIC_F_MOMENTS) {
        const size_t nb = (size_t)c->nph;
        c->mom[0] = (double*)dev_alloc(c, sizeof(double) * 4 * nodes * nb);
        c->mom[1] = (double*)dev_alloc(c, sizeof(double) * 4 * nodes * nb);
        c->mphi = (double*)dev_alloc(c, sizeof(double) * nodes * nb);
        c->mke[0] = (double*)dev_alloc(c, sizeof(double) * nodes * nb);
        c->mke[1] = (double*)dev_alloc(c, sizeof(double) * nodes * nb);
        c->d_bin = (int*)dev_alloc(c, sizeof(int));
        c->d_bsteps = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * nb);
        c->d_oml = (double*)dev_alloc(c, sizeof(double) * 6 * (size_t)std::max(c->ng, 1));
        if (c->prec == PIC_MIXED) {
            c->mom32[0] = (float*)dev_alloc(c, sizeof(float) * 5 * nodes);
            c->mom32[1] = (float*)dev_alloc(c, sizeof(float) * 5 * nodes);
            ok = ok && c->mom32[0] && c->mom32[1];
        }
        ok = ok && c->mom[0] && c->mom[1] && c->mphi && c->mke[0] && c->mke[1] && c->d_bin && c->d_bsteps && c->d_oml;
        if (c->nfine) {
            c->fine[0] = (double*)dev_alloc(c, sizeof(double) * 4 * c->nfine);
            c->fine[1] = (double*)dev_alloc(c, sizeof(double) * 4 * c->nfine);
            ok = ok && c->fine[0] && c->fine[1];
        }
    }
    ok = ok && c->d_step && c->d_iters && c->d_res && c->d_solve_flag && c->d_iter_total && c->d_vb_last;
    ok = ok && c->d_nslot && c->d_cnt && c->d_live && c->d_err && c->d_nch && c->d_next_id && c->d_child && c->rq && c->phi &&
         c->phi_alt && c->f64 && (c->e32 || c->e64) && c->d_norm && c->xs64 && c->xs32 && c->gpos && c->grad &&
         c->gcell && c->gq && c->gabs && c->gtab && c->gtab32 && c->gq32 && c->goff32 && c->gr2_32 && c->cell_ng &&
         c->cell_g && c->cursor;
    if (!ok || !sort_scratch_setup(c) || mg_setup(c) != PIC_OK) {
        destroy(c);
        return fail(nullptr, PIC_ENOMEM, "device allocation failed");
    }
    if (mixed && push32_set_window(c) != cudaSuccess) {
        destroy(c);
        return fail(nullptr, PIC_ECUDA, "push window size");
    }

    // ---- upload inputs
    // The caller's particle arrays are converted into the run's records on the
    // device (k_stage_particles, which also checks them).  Where the device reads
    // pageable host memory through the host's page tables (a coherent CPU-GPU
    // link), the kernel reads the arrays in place; elsewhere they go to device
    // scratch chunk by chunk first.
    unsigned int max_id = 0;
    bool any = false;
    unsigned long long nslot[2] = {(unsigned long long)run->n[0], (unsigned long long)run->n[1]};
    if (!t_ev && (run->n[0] > 0 || run->n[1] > 0)) {
        int dev = 0, pma = 0, ats = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, dev);
        cudaDeviceGetAttribute(&ats, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
        const bool direct = pma && ats && !(run->flags & PIC_F_STAGE_COPY);
        const int64_t nmax = std::max(run->n[0], run->n[1]);
        const int64_t chunk = direct ? nmax : std::min<int64_t>(nmax, (int64_t)1 << 24);
        unsigned int* flags = nullptr;   // [bad, largest id]
        double* sx = nullptr;
        double* sv = nullptr;
        uint32_t* sid = nullptr;
        cudaError_t e = cudaMalloc(&flags, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned int), c->stream);
        if (e == cudaSuccess && !direct) e = cudaMalloc(&sx, 3 * sizeof(double) * (size_t)chunk);
        if (e == cudaSuccess && !direct) e = cudaMalloc(&sv, 3 * sizeof(double) * (size_t)chunk);
        if (e == cudaSuccess && !direct) e = cudaMalloc(&sid, sizeof(uint32_t) * (size_t)chunk);
        for (int sp = 0; sp < 2 && e == cudaSuccess; ++sp)
            for (int64_t q0 = 0; q0 < run->n[sp] && e == cudaSuccess; q0 += chunk) {
                const int64_t m = std::min(chunk, run->n[sp] - q0);
                const double* x = run->x_host[sp] + 3 * q0;
                const double* v = run->v_host[sp] + 3 * q0;
                const uint32_t* id = run->id_host[sp] + q0;
                if (!direct) {
                    e = cudaMemcpyAsync(sx, x, 3 * sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, c->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(sv, v, 3 * sizeof(double) * (size_t)m, cudaMemcpyHostToDevice, c->stream);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(sid, id, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, c->stream);
                    x = sx;
                    v = sv;
                    id = sid;
                }
                if (e == cudaSuccess) launch_stage_particles(c, sp, x, v, id, m, q0, flags, flags + 1);
                if (e == cudaSuccess) e = cudaGetLastError();
                // the scratch is reused by the next chunk
                if (e == cudaSuccess && !direct) e = cudaStreamSynchronize(c->stream);
            }
        unsigned int hf[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(flags);
        cudaFree(sx);
        cudaFree(sv);
        cudaFree(sid);
        if (e != cudaSuccess) { destroy(c); return cuda_fail(nullptr, e, "particle upload"); }
        if (hf[0]) { destroy(c); return fail(nullptr, PIC_EINVAL, "run: particle outside the box or non-finite"); }
        max_id = hf[1];
        any = true;
    }
    const unsigned int next_id = t_ev ? (unsigned int)(run->n[0] + run->n[1]) : any ? max_id + 1 : 0;
    std::vector<float> xs32(5 * (size_t)c->n_xs);
    for (size_t i = 0; i < xs32.size(); ++i) xs32[i] = (float)gas->xs_host[i];
    std::vector<double> gpos(3 * ng1, 0.0), grad(ng1, 0.0);
    std::vector<float> goff(3 * ng1, 0.f), gr2(ng1, 0.f);
    for (int g = 0; g < c->ng; ++g) {
        for (int a = 0; a < 3; ++a) {
            gpos[3 * g + a] = grains->pos_host[3 * g + a];
            goff[3 * g + a] = (float)(grains->pos_host[3 * g + a] / mesh->dx - gcell[3 * g + a]);
        }
        grad[g] = grains->radius_host[g];
        gr2[g] = (float)((grad[g] / mesh->dx) * (grad[g] / mesh->dx));
    }
    gcell.resize(3 * ng1, 0);
    cudaError_t e = cudaSuccess;
    auto up = [&](void* d, const void* h, size_t b) {
        if (e == cudaSuccess && b) e = cudaMemcpy(d, h, b, cudaMemcpyHostToDevice);
    };
    up(c->d_nslot, nslot, sizeof nslot);
    up(c->d_next_id, &next_id, sizeof next_id);
    up(c->xs64, gas->xs_host, sizeof(double) * 5 * c->n_xs);
    up(c->xs32, xs32.data(), sizeof(float) * xs32.size());
    up(c->gpos, gpos.data(), sizeof(double) * gpos.size());
    up(c->grad, grad.data(), sizeof(double) * grad.size());
    up(c->gcell, gcell.data(), sizeof(int) * gcell.size());
    up(c->goff32, goff.data(), sizeof(float) * goff.size());
    up(c->gr2_32, gr2.data(), sizeof(float) * gr2.size());
    up(c->cell_ng, cell_ng.data(), sizeof(int) * cells);
    up(c->cell_g, cell_g.data(), sizeof(int) * cells * kMaxG);
    if (e == cudaSuccess) e = cudaMemset(c->d_cnt, 0, PIC_C_N * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_step, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_iters, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->d_res, 0, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(c->d_solve_flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_iter_total, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_vb_last, 0, sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(c->d_nch, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->gabs, 0, sizeof(unsigned long long) * 2 * ng1);
    if (e == cudaSuccess) e = cudaMemset(c->gq, 0, sizeof(double) * ng1);
    if (e == cudaSuccess) e = cudaMemset(c->gq32, 0, sizeof(float) * ng1);
    if (e == cudaSuccess) e = cudaMemset(c->phi, 0, sizeof(double) * nodes);
    if (e == cudaSuccess && (c->flags & PIC_F_MOMENTS)) {
        e = cudaMemset(c->d_bin, 0, sizeof(int));
        if (e == cudaSuccess) e = clear_moments(c, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess && t_ev) {
        // electrons take ids 0 .. n_e - 1, ions n_e .. n_e + n_i - 1
        launch_init_plasma(c, 0, run->n[0], 0u, t_ev[0]);
        launch_init_plasma(c, 1, run->n[1], (uint32_t)run->n[0], t_ev[1]);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { destroy(c); return cuda_fail(nullptr, e, "upload"); }

    // ---- unit-charge mesh field of each grain on its region nodes (Eq. 5), by
    // superposition: one solve per node plane that the grains' cell corners lie
    // on, for a unit charge on node (0, 0, k) of that plane (the mesh is periodic
    // in x and y, so a unit charge on node (i, j, k) gives the same potential
    // moved by (i, j)); each grain's table is then the sum of its 8 corners'
    // moved potentials with its CIC weights (launch_grain_tables_sup)
    {
        const double dx = mesh->dx;
        const double scale1 = ((1.0 / (dx * dx * dx)) * 0x1p-42) / kEPS0;
        std::vector<int> plane((size_t)nz + 1, -1), planes;
        for (int g = 0; g < c->ng; ++g)
            for (int dz = 0; dz < 2; ++dz) {
                const int k = gcell[3 * g + 2] + dz;
                if (plane[k] < 0) {
                    plane[k] = (int)planes.size();
                    planes.push_back(k);
                }
            }
        double* blk = nullptr;
        int* dplane = nullptr;
        cudaError_t eg = cudaSuccess;
        if (!planes.empty()) {
            eg = cudaMalloc(&blk, sizeof(double) * 343 * planes.size());
            if (eg == cudaSuccess) eg = cudaMalloc(&dplane, sizeof(int) * plane.size());
            if (eg == cudaSuccess)
                eg = cudaMemcpy(dplane, plane.data(), sizeof(int) * plane.size(), cudaMemcpyHostToDevice);
        }
        if (eg != cudaSuccess) {
            cudaFree(blk);
            cudaFree(dplane);
            destroy(c);
            return cuda_fail(nullptr, eg, "grain tables");
        }
        const unsigned long long unit = 1ull << 42;   // one elementary charge in the deposit's fixed point
        for (size_t q = 0; q < planes.size(); ++q) {
            cudaMemsetAsync(c->rq, 0, sizeof(unsigned long long) * nodes, c->stream);
            cudaMemcpyAsync(c->rq + (size_t)planes[q] * (size_t)nx * (size_t)ny, &unit, sizeof unit,
                            cudaMemcpyHostToDevice, c->stream);
            cudaMemsetAsync(c->phi, 0, sizeof(double) * nodes, c->stream);
            if (c->phi2) cudaMemsetAsync(c->phi2, 0, sizeof(float2) * nodes, c->stream);
            launch_rhs(c, scale1, 0.0, 0.0, false);
            int it = 0;
            double res = 0;
            const pic_status s = mg_solve(c, 0.0, 0.0, 1e-12, 200, &it, &res);
            if (s != PIC_OK) {
                cudaFree(blk);
                cudaFree(dplane);
                destroy(c);
                return fail(nullptr, s, "grain field solve did not converge");
            }
            phi_sync_f64(c);
            launch_green_block(c, planes[q], blk + (size_t)343 * q);
        }
        if (!planes.empty()) launch_grain_tables_sup(c, blk, dplane);
        eg = cudaStreamSynchronize(c->stream);
        cudaFree(blk);
        cudaFree(dplane);
        if (eg != cudaSuccess) { destroy(c); return cuda_fail(nullptr, eg, "grain tables"); }
        cudaMemsetAsync(c->gabs, 0, sizeof(unsigned long long) * 2 * ng1, c->stream);
        cudaMemsetAsync(c->phi, 0, sizeof(double) * nodes, c->stream);
        if (c->phi2) cudaMemsetAsync(c->phi2, 0, sizeof(float2) * 2 * nodes, c->stream);
        std::vector<double> tab(kTab * (size_t)ng1);
        e = cudaMemcpyAsync(tab.data(), c->gtab, sizeof(double) * tab.size(), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        std::vector<float> tab32(tab.size());
        for (size_t i = 0; i < tab.size(); ++i) tab32[i] = (float)tab[i];
        if (e == cudaSuccess) e = cudaMemcpy(c->gtab32, tab32.data(), sizeof(float) * tab32.size(),
                                             cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { destroy(c); return cuda_fail(nullptr, e, "grain tables"); }
    }

    // ---- cell order for the first steps, then rho_0 and phi_0
    sort_particles(c, 0);
    sort_particles(c, 1);
    c->parity ^= 1;
    cudaMemsetAsync(c->rq, 0, sizeof(unsigned long long) * nodes, c->stream);
    deposit_particles(c);
    launch_grains(c);
    const pic_status s = solve_now(c, c->tol, nullptr, nullptr);
    if (s != PIC_OK && s != PIC_ENOTCONV) {
        destroy(c);
        return fail(nullptr, s, "initial solve failed");
    }
    const pic_status k = check(c);
    if (k != PIC_OK) {
        std::string m = c->err;
        destroy(c);
        return fail(nullptr, k, m);
    }
    if (s == PIC_ENOTCONV) c->pending = PIC_ENOTCONV;
    *out = c;
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_init(const pic_mesh* mesh, const pic_electrodes* el, const pic_gas* gas, const pic_grains* grains,
                    const pic_run* run, void* cuda_stream, pic_ctx** out)
{
    return init_run(mesh, el, gas, grains, run, nullptr, cuda_stream, out);
}

pic_status pic_init_plasma(const pic_mesh* mesh, const pic_electrodes* el, const pic_gas* gas,
                           const pic_grains* grains, const pic_run* run, const double* t_ev, void* cuda_stream,
                           pic_ctx** out)
{
    g_init_error.clear();
    if (!t_ev) {
        if (out) *out = nullptr;
        return fail(nullptr, PIC_EINVAL, "t_ev is NULL");
    }
    return init_run(mesh, el, gas, grains, run, t_ev, cuda_stream, out);
}

pic_status pic_advance(pic_ctx* c)
{
    if (!c) return PIC_EINVAL;
    const bool mixed = c->prec == PIC_MIXED;
    cudaMemsetAsync(c->rq, 0, sizeof(unsigned long long) * c->nodes, c->stream);
    if (mixed) launch_efield32(c);
    else launch_efield64(c);
    cudaEvent_t ev = prof_begin(c);
    if (mixed) launch_push32(c);
    else launch_push64(c);
    prof_end(c, ev, true);
    if (mixed) launch_children32(c);
    else launch_children64(c);
    if (c->flags & PIC_F_COULOMB) launch_coulomb(c);
    if (c->eepf) {
        launch_eepf(c);
        c->eepf_steps += 1;
    }
    launch_grains(c);
    c->step += 1;
    if (c->sort_every > 0 && c->step % c->sort_every == 0) {
        sort_particles(c, 0);
        sort_particles(c, 1);
        c->parity ^= 1;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "advance launch");
    return PIC_OK;
}

}  // extern "C"

namespace {

// Capture what `enqueue` queues on c->stream into an executable graph, on the
// private capture stream; the host-side launch counter and particle buffer
// pointers are restored, and the graph's kernel count returned in *kernels.
template <class F>
cudaGraphExec_t capture(pic_ctx* c, int* kernels, F&& enqueue)
{
    cudaStream_t user = c->stream;
    const int prof = c->prof;
    const int64_t l0 = c->launches;
    void* keep[8] = {c->pos[0], c->pos[1], c->vel[0], c->vel[1], c->pos_alt[0], c->pos_alt[1], c->vel_alt[0],
                     c->vel_alt[1]};
    c->stream = c->cap_stream;
    c->prof = 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        enqueue();
        if (cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && g) {
            if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
            cudaGraphDestroy(g);
        }
    }
    *kernels = (int)(c->launches - l0);
    c->launches = l0;
    c->stream = user;
    c->prof = prof;
    c->pos[0] = (void*)keep[0]; c->pos[1] = keep[1]; c->vel[0] = keep[2]; c->vel[1] = keep[3];
    c->pos_alt[0] = keep[4]; c->pos_alt[1] = keep[5]; c->vel_alt[0] = keep[6]; c->vel_alt[1] = keep[7];
    return ex;
}

// The solve graph: head (rhs, starting residual, first decision) followed by a
// conditional while node whose body is one refinement iteration.
cudaGraphExec_t capture_solve(pic_ctx* c)
{
    cudaStream_t user = c->stream;
    const int prof = c->prof;
    const int64_t l0 = c->launches;
    c->stream = c->cap_stream;
    c->prof = 0;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    cudaGraphConditionalHandle h{};
    ok = ok && cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
    std::vector<cudaGraphNode_t> frontier;
    if (ok && cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                  cudaSuccess) {
        enqueue_solve_head(c, c->tol, c->max_cycles, h);
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if (cudaStreamGetCaptureInfo(c->cap_stream, &st, nullptr, nullptr, &deps, nullptr, &nd) == cudaSuccess)
            frontier.assign(deps, deps + nd);
        ok = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && !frontier.empty();
    } else {
        ok = false;
    }
    c->n_solve_head = (int)(c->launches - l0);
    if (ok) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        ok = cudaGraphAddNode(&cn, g, frontier.data(), nullptr, frontier.size(), &cp) == cudaSuccess;
        if (ok) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            const int64_t l1 = c->launches;
            ok = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
            if (ok) {
                enqueue_solve_iteration(c, c->tol, c->max_cycles, h);
                ok = cudaStreamEndCapture(c->cap_stream, &body) == cudaSuccess;
            }
            c->n_solve_body = (int)(c->launches - l1);
        }
        // after the loop
        if (ok) {
            const int64_t l2 = c->launches;
            ok = cudaStreamBeginCaptureToGraph(c->cap_stream, g, &cn, nullptr, 1, cudaStreamCaptureModeThreadLocal) ==
                 cudaSuccess;
            if (ok) {
                enqueue_solve_tail(c);
                ok = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess;
            }
            c->n_solve_head += (int)(c->launches - l2);
        }
    }
    if (ok && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    if (g) cudaGraphDestroy(g);
    c->launches = l0;
    c->stream = user;
    c->prof = prof;
    return ex;
}

pic_status ensure_graphs(pic_ctx* c, bool sort)
{
    const bool mixed = c->prec == PIC_MIXED;
    const int p = c->parity, so = sort ? 1 : 0;
    if (!c->g_pre)
        c->g_pre = capture(c, &c->n_pre, [&] {
            cudaMemsetAsync(c->rq, 0, sizeof(unsigned long long) * c->nodes, c->stream);
            if (mixed) launch_efield32(c);
            else launch_efield64(c);
        });
    if (!c->g_push[p])
        c->g_push[p] = capture(c, &c->n_push, [&] {
            if (mixed) launch_push32(c);
            else launch_push64(c);
        });
    if (!c->g_post[p][so])
        c->g_post[p][so] = capture(c, &c->n_post[so], [&] {
            if (mixed) launch_children32(c);
            else launch_children64(c);
            if (c->flags & PIC_F_COULOMB) launch_coulomb(c);
            if (c->eepf) launch_eepf(c);
            launch_grains(c);
            if (sort) {
                sort_particles(c, 0);
                sort_particles(c, 1);
            }
        });
    if (!c->g_solve) c->g_solve = capture_solve(c);
    if (!c->g_pre || !c->g_push[p] || !c->g_post[p][so] || !c->g_solve)
        return fail(c, PIC_ECUDA, "CUDA graph capture failed");
    return PIC_OK;
}

// the moment sample reads the particle buffers of the parity after the step's
// sort, so its graph is captured for that parity when it is first needed
pic_status ensure_mom_graph(pic_ctx* c)
{
    const int p = c->parity;
    if (!c->g_mom[p]) c->g_mom[p] = capture(c, &c->n_mom, [&] { launch_moments_all(c); });
    return c->g_mom[p] ? PIC_OK : fail(c, PIC_ECUDA, "CUDA graph capture failed");
}

pic_status launch_solve_graph(pic_ctx* c)
{
    cudaEvent_t ev = prof_begin(c);
    const cudaError_t e = cudaGraphLaunch(c->g_solve, c->stream);
    prof_end(c, ev, false);
    c->launches += c->n_solve_head;
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "solve graph launch");
}

}  // namespace

extern "C" {

pic_status pic_solve(pic_ctx* c, int32_t* iterations, double* rel_residual)
{
    if (!c) return PIC_EINVAL;
    pic_status k = ensure_graphs(c, false);
    if (k != PIC_OK) return k;
    k = launch_solve_graph(c);
    if (k != PIC_OK) return k;
    unsigned int it = 0;
    double res = 0.0;
    const pic_status chk = check(c);
    cudaMemcpy(&it, c->d_iters, sizeof it, cudaMemcpyDeviceToHost);
    cudaMemcpy(&res, c->d_res, sizeof res, cudaMemcpyDeviceToHost);
    if (iterations) *iterations = (int32_t)it;
    if (rel_residual) *rel_residual = res;
    c->last_iters = it;
    c->last_res = res;
    return chk;
}

}  // extern "C"

namespace {

// queue n steps on the run's stream; no final synchronisation
pic_status step_enqueue(pic_ctx* c, int32_t n_steps)
{
    if (c->pending != PIC_OK) {
        const pic_status p = c->pending;
        c->pending = PIC_OK;
        return fail(c, p, "an earlier solve did not converge");
    }
    if (c->flags & PIC_F_NO_GRAPH) {
        for (int32_t s = 0; s < n_steps; ++s) {
            pic_status r = pic_advance(c);
            if (r != PIC_OK) return r;
            int it = 0;
            double res = 0.0;
            r = solve_now(c, c->tol, &it, &res);
            if (r == PIC_ENOTCONV) c->pending = PIC_ENOTCONV;
            else if (r != PIC_OK) return fail(c, r, "Poisson solve failed");
            if (c->flags & PIC_F_MOMENTS) {
                launch_moments_all(c);
                c->msteps += 1;
            }
        }
        return PIC_OK;
    }
    for (int32_t s = 0; s < n_steps; ++s) {
        const bool sort = c->sort_every > 0 && (c->step + 1) % c->sort_every == 0;
        pic_status r = ensure_graphs(c, sort);
        if (r != PIC_OK) return r;
        const int p = c->parity;
        cudaError_t e = cudaGraphLaunch(c->g_pre, c->stream);
        cudaEvent_t ev = prof_begin(c);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->g_push[p], c->stream);
        prof_end(c, ev, true);
        if (e == cudaSuccess) e = cudaGraphLaunch(c->g_post[p][sort ? 1 : 0], c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "step graph launch");
        c->launches += c->n_pre + c->n_push + c->n_post[sort ? 1 : 0];
        if (c->eepf) c->eepf_steps += 1;
        c->step += 1;
        if (sort) {
            std::swap(c->pos[0], c->pos_alt[0]);
            std::swap(c->pos[1], c->pos_alt[1]);
            std::swap(c->vel[0], c->vel_alt[0]);
            std::swap(c->vel[1], c->vel_alt[1]);
            c->parity ^= 1;
        }
        r = launch_solve_graph(c);
        if (r != PIC_OK) return r;
        if (c->flags & PIC_F_MOMENTS) {
            r = ensure_mom_graph(c);
            if (r != PIC_OK) return r;
            e = cudaGraphLaunch(c->g_mom[c->parity], c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "moments graph launch");
            c->launches += c->n_mom;
            c->msteps += 1;
        }
    }
    return PIC_OK;
}

// the step graphs (not the solve): rebuilt on the next step
void drop_graphs(pic_ctx* c)
{
    cudaGraphExec_t* gs[] = {&c->g_push[0], &c->g_push[1], &c->g_post[0][0], &c->g_post[0][1], &c->g_post[1][0],
                             &c->g_post[1][1], &c->g_mom[0], &c->g_mom[1]};
    for (cudaGraphExec_t* g : gs)
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
}


size_t tuning_window_bytes(const int32_t tile[3], int32_t halo)
{
    return sizeof(unsigned long long) * (size_t)(tile[0] + 1 + 2 * halo) * (size_t)(tile[1] + 1 + 2 * halo) *
           (size_t)(tile[2] + 1 + 2 * halo);
}

// cache key: device name, mesh, particle count (2 significant digits), precision
std::string tuning_key(const pic_ctx* c)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (char& ch : name)
        if (ch == '"' || ch == '|' || ch == '\\') ch = '_';
    unsigned long long ns[2] = {0, 0};
    cudaMemcpy(ns, c->d_nslot, sizeof ns, cudaMemcpyDeviceToHost);
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|%dx%dx%d|%.1e|%s", name.c_str(), c->nx, c->ny, c->nz,
                  (double)(ns[0] + ns[1]), c->prec == PIC_MIXED ? "mixed" : "fp64");
    return buf;
}

}  // namespace

struct pic_batch {
    std::vector<pic_ctx*> runs;
    std::vector<cudaStream_t> streams;
};

extern "C" {

pic_status pic_step(pic_ctx* c, int32_t n_steps)
{
    if (!c || n_steps < 0) return PIC_EINVAL;
    const pic_status r = step_enqueue(c, n_steps);
    if (r != PIC_OK) return r;
    return check(c);
}

pic_status pic_tune_sort(pic_ctx* c, int32_t steps_per_candidate, int32_t* chosen)
{
    if (!c || steps_per_candidate < 1) return PIC_EINVAL;
    const int32_t cand[] = {2, 3, 4, 5, 6, 8, 10, 14, 20};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!PIC_CUDA_OK(cudaEventCreate(&e0)) || !PIC_CUDA_OK(cudaEventCreate(&e1))) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "tune events");
    }
    int32_t best = c->sort_every;
    float best_ms = 0.f;
    pic_status st = PIC_OK;
    for (int32_t s : cand) {
        c->sort_every = s;
        const int32_t whole = std::max(steps_per_candidate, 2 * s);
        const int32_t n = (whole + s - 1) / s * s;
        // start on a sort boundary so that every candidate covers whole periods
        const int32_t lead = (int32_t)((s - c->step % s) % s);
        if (lead > 0 && (st = step_enqueue(c, lead)) != PIC_OK) break;
        cudaEventRecord(e0, c->stream);
        if ((st = step_enqueue(c, n)) != PIC_OK) break;
        cudaEventRecord(e1, c->stream);
        if ((st = check(c)) != PIC_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= (float)n;
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best = s;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sort_every = best;
    if (chosen) *chosen = best;
    return st;
}

pic_status pic_get_tuning(const pic_ctx* c, pic_tuning* out)
{
    if (!c || !out) return PIC_EINVAL;
    out->sort_every = c->sort_every;
    for (int a = 0; a < 3; ++a) out->tile[a] = c->tile[a];
    out->halo = c->halo;
    out->order = c->sort_order;
    return PIC_OK;
}

pic_status pic_set_tuning(pic_ctx* c, const pic_tuning* t)
{
    if (!c || !t) return PIC_EINVAL;
    if (t->sort_every < 1 || t->sort_every > 1000) return fail(c, PIC_EINVAL, "tuning: sort_every in [1, 1000]");
    if (c->prec != PIC_MIXED) {
        c->sort_every = t->sort_every;
        return PIC_OK;
    }
    const int n[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; ++a)
        if (t->tile[a] < 1 || t->tile[a] > n[a] || t->tile[a] > 64)
            return fail(c, PIC_EINVAL, "tuning: tile edges in [1, min(mesh, 64)]");
    if (t->halo < 0 || t->halo > 8) return fail(c, PIC_EINVAL, "tuning: halo in [0, 8]");
    if (t->order < 0 || t->order > 2)
        return fail(c, PIC_EINVAL, "tuning: order 0 (cell), 1 (tile) or 2 (2x2x2-cell blocks)");
    if (tuning_window_bytes(t->tile, t->halo) > kMaxWindowBytes)
        return fail(c, PIC_EINVAL, "tuning: the deposit window (tile + 1 + 2 halo nodes per axis, 8 B each) "
                                   "exceeds 96 KB");
    c->sort_every = t->sort_every;
    const bool same = t->tile[0] == c->tile[0] && t->tile[1] == c->tile[1] && t->tile[2] == c->tile[2] &&
                      t->halo == c->halo && t->order == c->sort_order;
    if (same) return PIC_OK;
    // new sort keys: wait for queued work, size the key buffers, re-sort both
    // species now (the tile ranges must describe the new order), drop the step
    // graphs (grid and window size are baked into them)
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning sync");
    int ntile[3];
    for (int a = 0; a < 3; ++a) ntile[a] = (n[a] + t->tile[a] - 1) / t->tile[a];
    const int64_t ntiles = (int64_t)ntile[0] * ntile[1] * ntile[2];
    const size_t nkeys = (size_t)ntiles * (size_t)(t->tile[0] * t->tile[1] * t->tile[2]);
    if (nkeys > c->nkeys_cap || ntiles > c->ntiles_cap) {
        unsigned int* cur = nkeys > c->nkeys_cap ? (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (nkeys + 1))
                                                 : c->cursor;
        unsigned int* ts0 = ntiles > c->ntiles_cap ? (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (ntiles + 1))
                                                   : c->tstart[0];
        unsigned int* ts1 = ntiles > c->ntiles_cap ? (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (ntiles + 1))
                                                   : c->tstart[1];
        if (!cur || !ts0 || !ts1) return fail(c, PIC_ENOMEM, "tuning: key buffers");
        c->cursor = cur;
        c->tstart[0] = ts0;
        c->tstart[1] = ts1;
        c->nkeys_cap = std::max(c->nkeys_cap, nkeys);
        c->ntiles_cap = std::max(c->ntiles_cap, ntiles);
        const size_t old_keys = c->nkeys;
        c->nkeys = nkeys;
        if (nkeys > old_keys && !sort_scratch_setup(c)) return fail(c, PIC_ENOMEM, "tuning: scan scratch");
    }
    for (int a = 0; a < 3; ++a) { c->tile[a] = t->tile[a]; c->ntile[a] = ntile[a]; }
    c->ntiles = ntiles;
    c->nkeys = nkeys;
    c->halo = t->halo;
    c->sort_order = t->order;
    e = push32_set_window(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning: push window size");
    drop_graphs(c);
    sort_particles(c, 0);
    sort_particles(c, 1);
    c->parity ^= 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "tuning re-sort");
    return check(c);
}

pic_status pic_tune(pic_ctx* c, int32_t steps_per_candidate, const char* cache_path, pic_tuning* chosen)
{
    if (!c || steps_per_candidate < 1) return PIC_EINVAL;
    const std::string key = tuning_key(c);
    pic_tuning best{};
    pic_get_tuning(c, &best);
    if (cache_path && pic_tune_cache_load(cache_path, key.c_str(), &best) == PIC_OK) {
        const pic_status st = pic_set_tuning(c, &best);
        if (st == PIC_OK && chosen) *chosen = best;
        return st;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!PIC_CUDA_OK(cudaEventCreate(&e0)) || !PIC_CUDA_OK(cudaEventCreate(&e1))) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(c, cudaGetLastError(), "tune events");
    }
    // ms per step of one candidate over whole sort periods, after a warm-up period
    pic_status st = PIC_OK;
    auto time_it = [&](const pic_tuning& t, float* ms) -> pic_status {
        pic_status r = pic_set_tuning(c, &t);
        if (r != PIC_OK) return r;
        const int32_t s = t.sort_every;
        const int32_t lead = (int32_t)((s - c->step % s) % s) + s;
        if ((r = step_enqueue(c, lead)) != PIC_OK) return r;
        const int32_t n = (std::max(steps_per_candidate, 2 * s) + s - 1) / s * s;
        cudaEventRecord(e0, c->stream);
        if ((r = step_enqueue(c, n)) != PIC_OK) return r;
        cudaEventRecord(e1, c->stream);
        if ((r = check(c)) != PIC_OK) return r;
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= (float)n;
        return PIC_OK;
    };
    float best_ms = 0.f;
    // coordinate search: tile shape, then window margin, then sort order, then
    // sort interval
    if (c->prec == PIC_MIXED) {
        const int shapes[][3] = {{8, 8, 8}, {16, 8, 4}, {8, 8, 4}, {16, 8, 8}, {16, 16, 4}, {32, 8, 4}};
        for (const auto& sh : shapes) {
            pic_tuning t = best;
            for (int a = 0; a < 3; ++a) t.tile[a] = std::min(sh[a], a == 0 ? c->nx : a == 1 ? c->ny : c->nz);
            if (tuning_window_bytes(t.tile, t.halo) > kMaxWindowBytes) continue;
            float ms = 0.f;
            if ((st = time_it(t, &ms)) != PIC_OK) break;
            if (best_ms == 0.f || ms < best_ms) { best_ms = ms; best = t; }
        }
        for (int h = 1; h <= 3 && st == PIC_OK; ++h) {
            if (h == best.halo) continue;
            pic_tuning t = best;
            t.halo = h;
            if (tuning_window_bytes(t.tile, t.halo) > kMaxWindowBytes) continue;
            float ms = 0.f;
            if ((st = time_it(t, &ms)) != PIC_OK) break;
            if (ms < best_ms) { best_ms = ms; best = t; }
        }
        const int32_t order0 = best.order;
        for (int32_t o = 0; o <= 2 && st == PIC_OK; ++o) {
            if (o == order0) continue;
            pic_tuning t = best;
            t.order = o;
            float ms = 0.f;
            st = time_it(t, &ms);
            if (st == PIC_OK && ms < best_ms) { best_ms = ms; best = t; }
        }
    }
    const int32_t sorts[] = {2, 3, 4, 5, 6, 8, 10, 14, 20};
    for (int32_t sv : sorts) {
        if (st != PIC_OK) break;
        pic_tuning t = best;
        t.sort_every = sv;
        float ms = 0.f;
        if ((st = time_it(t, &ms)) != PIC_OK) break;
        if (best_ms == 0.f || ms < best_ms) { best_ms = ms; best = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PIC_OK) return st;
    st = pic_set_tuning(c, &best);
    if (st != PIC_OK) return st;
    if (chosen) *chosen = best;
    if (cache_path && pic_tune_cache_store(cache_path, key.c_str(), &best) != PIC_OK)
        return fail(c, PIC_EINVAL, std::string("tuning cache not writable: ") + cache_path);
    return PIC_OK;
}

pic_status pic_batch_init(int32_t n, const pic_mesh* meshes, const pic_electrodes* els, const pic_gas* gases,
                          const pic_grains* grains, const pic_run* runs, pic_batch** out)
{
    g_init_error.clear();
    if (!out || n < 1 || !meshes || !els || !gases || !grains || !runs)
        return fail(nullptr, PIC_EINVAL, "pic_batch_init: need n >= 1 and the five argument arrays");
    *out = nullptr;
    pic_batch* b = new (std::nothrow) pic_batch();
    if (!b) return fail(nullptr, PIC_ENOMEM, "host allocation");
    for (int32_t r = 0; r < n; ++r) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        pic_ctx* c = nullptr;
        pic_status st = e == cudaSuccess ? pic_init(meshes + r, els + r, gases + r, grains + r, runs + r, s, &c)
                                         : PIC_ECUDA;
        if (st != PIC_OK) {
            const std::string m = "run " + std::to_string(r) + ": " +
                                  (e == cudaSuccess ? g_init_error : std::string(cudaGetErrorString(e)));
            if (s) cudaStreamDestroy(s);
            pic_batch_destroy(b);
            return fail(nullptr, st, m);
        }
        b->runs.push_back(c);
        b->streams.push_back(s);
    }
    *out = b;
    return PIC_OK;
}

pic_status pic_batch_step(pic_batch* b, int32_t n_steps)
{
    if (!b || n_steps < 0) return PIC_EINVAL;
    pic_status first = PIC_OK;
    // one step of every run at a time, so the runs advance side by side
    for (int32_t s = 0; s < n_steps && first == PIC_OK; ++s)
        for (pic_ctx* c : b->runs) {
            const pic_status r = step_enqueue(c, 1);
            if (r != PIC_OK && first == PIC_OK) first = r;
        }
    for (pic_ctx* c : b->runs) {
        const pic_status r = check(c);
        if (r != PIC_OK && first == PIC_OK) first = r;
    }
    return first;
}

pic_ctx* pic_batch_run(pic_batch* b, int32_t r)
{
    if (!b || r < 0 || r >= (int32_t)b->runs.size()) return nullptr;
    return b->runs[r];
}

void pic_batch_destroy(pic_batch* b)
{
    if (!b) return;
    for (pic_ctx* c : b->runs) pic_destroy(c);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    delete b;
}

pic_status pic_grain_charges(pic_ctx* c, int64_t* n_abs_host, double* q_host)
{
    if (!c) return PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (c->ng == 0) return PIC_OK;
    cudaError_t e = cudaSuccess;
    if (n_abs_host) e = cudaMemcpy(n_abs_host, c->gabs, sizeof(int64_t) * 2 * c->ng, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && q_host) e = cudaMemcpy(q_host, c->gq, sizeof(double) * c->ng, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "grain copy");
}

namespace {
// copy the slots of one species to the host and keep the live ones, in SI
pic_status fetch(pic_ctx* c, int sp, std::vector<double>& x, std::vector<double>& v, std::vector<uint32_t>& id)
{
    unsigned long long ns[2];
    cudaError_t e = cudaMemcpy(ns, c->d_nslot, sizeof ns, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "slot count");
    const size_t n = (size_t)ns[sp];
    x.clear(); v.clear(); id.clear();
    if (c->prec == PIC_MIXED) {
        std::vector<float4> P(n), V(n);
        e = cudaMemcpy(P.data(), c->pos[sp], sizeof(float4) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(V.data(), c->vel[sp], sizeof(float4) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "particle copy");
        const double vs = c->dx / c->dt;
        for (size_t q = 0; q < n; ++q) {
            int cell;
            std::memcpy(&cell, &P[q].w, 4);
            if (cell < 0) continue;
            const int i = cell & 1023, j = (cell >> 10) & 1023, k = cell >> 20;
            x.push_back((i + (double)P[q].x) * c->dx);
            x.push_back((j + (double)P[q].y) * c->dx);
            x.push_back((k + (double)P[q].z) * c->dx);
            v.push_back(V[q].x * vs); v.push_back(V[q].y * vs); v.push_back(V[q].z * vs);
            uint32_t u;
            std::memcpy(&u, &V[q].w, 4);
            id.push_back(u);
        }
    } else {
        std::vector<double4> P(n), V(n);
        e = cudaMemcpy(P.data(), c->pos[sp], sizeof(double4) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(V.data(), c->vel[sp], sizeof(double4) * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "particle copy");
        for (size_t q = 0; q < n; ++q) {
            if (P[q].w < 0.0) continue;
            x.push_back(P[q].x); x.push_back(P[q].y); x.push_back(P[q].z);
            v.push_back(V[q].x); v.push_back(V[q].y); v.push_back(V[q].z);
            id.push_back((uint32_t)V[q].w);
        }
    }
    return PIC_OK;
}
}  // namespace

pic_status pic_counts(pic_ctx* c, int64_t* n_live, int64_t* counters)
{
    if (!c) return PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (n_live) {
        // counted on the device (the records stay there)
        count_live(c);
        unsigned long long h[2] = {0, 0};
        cudaError_t e = cudaMemcpyAsync(h, c->d_live, sizeof h, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "live count");
        n_live[0] = (int64_t)h[0];
        n_live[1] = (int64_t)h[1];
    }
    if (counters) {
        const cudaError_t e = cudaMemcpy(counters, c->d_cnt, sizeof(int64_t) * PIC_C_N, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "counters");
    }
    return PIC_OK;
}

pic_status pic_get_particles(pic_ctx* c, int32_t sp, double* x_host, double* v_host, uint32_t* id_host, int64_t cap,
                             int64_t* n_out)
{
    if (!c || sp < 0 || sp > 1) return PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    std::vector<double> x, v;
    std::vector<uint32_t> id;
    k = fetch(c, sp, x, v, id);
    if (k != PIC_OK) return k;
    if (n_out) *n_out = (int64_t)id.size();
    if ((int64_t)id.size() > cap) return fail(c, PIC_EINVAL, "particle buffer too small");
    if (x_host) std::memcpy(x_host, x.data(), sizeof(double) * x.size());
    if (v_host) std::memcpy(v_host, v.data(), sizeof(double) * v.size());
    if (id_host) std::memcpy(id_host, id.data(), sizeof(uint32_t) * id.size());
    return PIC_OK;
}

pic_status pic_get_rho(pic_ctx* c, int64_t* rq, size_t len)
{
    if (!c || !rq || len != c->nodes) return c ? fail(c, PIC_EINVAL, "rho length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    const cudaError_t e = cudaMemcpy(rq, c->rq, sizeof(int64_t) * len, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "rho copy");
}

pic_status pic_get_phi(pic_ctx* c, double* phi, size_t len)
{
    if (!c || !phi || len != c->nodes) return c ? fail(c, PIC_EINVAL, "phi length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    phi_sync_f64(c);
    cudaError_t e = cudaMemcpyAsync(phi, c->phi, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "phi copy");
}

pic_status pic_set_phi(pic_ctx* c, const double* phi, size_t len)
{
    if (!c || !phi || len != c->nodes) return c ? fail(c, PIC_EINVAL, "phi length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    cudaError_t e = cudaMemcpyAsync(c->phi, phi, sizeof(double) * len, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) phi_from_f64(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "phi copy");
}

pic_status pic_get_grain_table(pic_ctx* c, double* tab, size_t len)
{
    if (!c || (len && !tab) || len != (size_t)kTab * c->ng) return c ? fail(c, PIC_EINVAL, "table length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK || !len) return k;
    const cudaError_t e = cudaMemcpy(tab, c->gtab, sizeof(double) * len, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "table copy");
}

pic_status pic_set_grain_table(pic_ctx* c, const double* tab, size_t len)
{
    if (!c || (len && !tab) || len != (size_t)kTab * c->ng) return c ? fail(c, PIC_EINVAL, "table length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK || !len) return k;
    std::vector<float> t32(len);
    for (size_t i = 0; i < len; ++i) t32[i] = (float)tab[i];
    cudaError_t e = cudaMemcpy(c->gtab, tab, sizeof(double) * len, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->gtab32, t32.data(), sizeof(float) * len, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "table copy");
}

pic_status pic_set_grain_counts(pic_ctx* c, const int64_t* n_abs, size_t len)
{
    if (!c || (len && !n_abs) || len != (size_t)2 * c->ng) return c ? fail(c, PIC_EINVAL, "count length") : PIC_EINVAL;
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (len) {
        for (size_t i = 0; i < len; ++i)
            if (n_abs[i] < 0) return fail(c, PIC_EINVAL, "negative count");
        const cudaError_t e = cudaMemcpy(c->gabs, n_abs, sizeof(int64_t) * len, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "count copy");
    }
    cudaMemsetAsync(c->rq, 0, sizeof(unsigned long long) * c->nodes, c->stream);
    deposit_particles(c);
    launch_grains(c);
    return pic_solve(c, nullptr, nullptr);
}

pic_status pic_profile(pic_ctx* c, int32_t enable)
{
    if (!c) return PIC_EINVAL;
    const pic_status k = check(c);
    if (k != PIC_OK) return k;
    drop_events(c);
    c->prof = enable ? 1 : 0;
    const cudaError_t e = cudaMemcpy(&c->prof_iter0, c->d_iter_total, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? PIC_OK : cuda_fail(c, e, "iteration counter");
}

pic_status pic_profile_read(pic_ctx* c, double* push_ms, int64_t* push_launches, double* solve_ms, int64_t* solves,
                            int64_t* solve_iterations, int64_t* kernels_launched)
{
    if (!c) return PIC_EINVAL;
    const pic_status k = check(c);
    if (k != PIC_OK) return k;
    double t[2] = {0.0, 0.0};
    int idx = 0;
    for (auto* v : {&c->ev_push, &c->ev_solve}) {
        for (auto& pr : *v) {
            float ms = 0.f;
            const cudaError_t e = cudaEventElapsedTime(&ms, pr.first, pr.second);
            if (e != cudaSuccess) return cuda_fail(c, e, "event time");
            t[idx] += ms;
        }
        ++idx;
    }
    unsigned long long tot = 0;
    const cudaError_t e = cudaMemcpy(&tot, c->d_iter_total, sizeof tot, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "iteration counter");
    if (push_ms) *push_ms = t[0];
    if (push_launches) *push_launches = (int64_t)c->ev_push.size() * 2;   // one launch per species
    if (solve_ms) *solve_ms = t[1];
    if (solves) *solves = (int64_t)c->ev_solve.size();
    if (solve_iterations) *solve_iterations = (int64_t)(tot - c->prof_iter0);
    if (kernels_launched) *kernels_launched = c->launches + (int64_t)tot * c->n_solve_body;
    return PIC_OK;
}

pic_status pic_eepf(pic_ctx* c, int64_t* counts, size_t len, int64_t* steps, int32_t reset)
{
    if (!c) return PIC_EINVAL;
    if (!c->eepf) return fail(c, PIC_EINVAL, "the energy histogram is off (eepf_bins = 0)");
    if (!counts || len != (size_t)c->nz * (c->eepf_bins + 1)) return fail(c, PIC_EINVAL, "eepf length");
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    cudaError_t e = cudaMemcpyAsync(counts, c->eepf, sizeof(int64_t) * len, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && reset) e = cudaMemsetAsync(c->eepf, 0, sizeof(int64_t) * len, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "eepf copy");
    if (steps) *steps = c->eepf_steps;
    if (reset) c->eepf_steps = 0;
    return PIC_OK;
}

pic_status pic_moments(pic_ctx* c, int32_t what, double* out, size_t len, int32_t reset)
{
    if (!c) return PIC_EINVAL;
    if (!(c->flags & PIC_F_MOMENTS)) return fail(c, PIC_EINVAL, "moments need PIC_F_MOMENTS at init");
    if (what < 0 || what > 6) return fail(c, PIC_EINVAL, "moments: what in 0..6");
    if (!out || len != (what == 3 || what == 4 ? 3 : 1) * c->nodes) return fail(c, PIC_EINVAL, "moments length");
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (c->msteps == 0) return fail(c, PIC_EINVAL, "moments: empty window");
    k = moments_window(c, what, 0, c->nph, c->msteps, out);
    if (k != PIC_OK) return k;
    if (reset) {
        const cudaError_t e = clear_moments(c, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "moments reset");
        c->msteps = 0;
    }
    return check(c);
}

pic_status pic_moments_phase(pic_ctx* c, int32_t what, int32_t bin, double* out, size_t len, int64_t* steps_out)
{
    if (!c) return PIC_EINVAL;
    if (!(c->flags & PIC_F_MOMENTS)) return fail(c, PIC_EINVAL, "moments need PIC_F_MOMENTS at init");
    if (what < 0 || what > 6 || bin < 0 || bin >= c->nph)
        return fail(c, PIC_EINVAL, "moments_phase: what in 0..6, bin in [0, mom_phases)");
    if (!out || len != (what == 3 || what == 4 ? 3 : 1) * c->nodes) return fail(c, PIC_EINVAL, "moments length");
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    int64_t steps = c->msteps;
    if (c->nph > 1) {
        unsigned long long n = 0;
        const cudaError_t e = cudaMemcpy(&n, c->d_bsteps + bin, sizeof n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "moments copy");
        steps = (int64_t)n;
    }
    if (steps_out) *steps_out = steps;
    if (steps == 0) return fail(c, PIC_EINVAL, "moments_phase: no samples in this bin");
    return moments_window(c, what, bin, bin + 1, steps, out);
}

pic_status pic_oml_charges(pic_ctx* c, int32_t with_cx, double* out, size_t len)
{
    if (!c) return PIC_EINVAL;
    if (!(c->flags & PIC_F_MOMENTS)) return fail(c, PIC_EINVAL, "oml_charges needs PIC_F_MOMENTS at init");
    if ((c->ng > 0 && !out) || len != 6 * (size_t)c->ng) return fail(c, PIC_EINVAL, "oml_charges length");
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (c->msteps == 0) return fail(c, PIC_EINVAL, "moments: empty window");
    if (c->ng == 0) return PIC_OK;
    launch_oml(c, with_cx != 0, c->d_oml);
    cudaError_t e = cudaMemcpyAsync(out, c->d_oml, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "oml_charges");
    return check(c);
}

pic_status pic_fine_moments(pic_ctx* c, int32_t what, double* out, size_t len)
{
    if (!c) return PIC_EINVAL;
    if (!c->nfine) return fail(c, PIC_EINVAL, "the fine grid is off (fine_n = 0)");
    if (what < 1 || what > 4) return fail(c, PIC_EINVAL, "fine_moments: what in 1..4");
    if (!out || len != (what >= 3 ? 3 : 1) * c->nfine) return fail(c, PIC_EINVAL, "fine_moments length");
    pic_status k = check(c);
    if (k != PIC_OK) return k;
    if (c->msteps == 0) return fail(c, PIC_EINVAL, "moments: empty window");
    std::vector<double> m(4 * c->nfine);
    const cudaError_t e = cudaMemcpy(m.data(), c->fine[(what - 1) % 2], sizeof(double) * m.size(),
                                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "fine moments copy");
    const double h = c->fine_h;
    const double norm = c->W / ((h * h * h) * (double)c->msteps);
    for (size_t q = 0; q < c->nfine; ++q) {
        if (what <= 2) out[q] = m[4 * q] * norm;
        else
            for (int a = 0; a < 3; ++a) out[3 * q + a] = m[4 * q + 1 + a] * norm;
    }
    return PIC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tuning cache: a JSON object with one member per line,
//   "<device>|<nx>x<ny>x<nz>|<particles>|<precision>": {"sort_every": S, "tile": [X, Y, Z], "halo": H, "order": O},
// read and rewritten whole by pic_tune_cache_store (last write wins).
extern "C" pic_status pic_tune_cache_load(const char* path, const char* key, pic_tuning* out)
{
    if (!path || !key || !out) return PIC_EINVAL;
    std::FILE* f = std::fopen(path, "r");
    if (!f) return PIC_EINVAL;
    const std::string want = std::string("\"") + key + "\":";
    char line[1024];
    pic_status st = PIC_EINVAL;
    while (std::fgets(line, sizeof line, f)) {
        const char* at = std::strstr(line, want.c_str());
        if (!at) continue;
        pic_tuning t{};
        t.order = 0;   // entries written before the sort order was a choice
        const int got = std::sscanf(at + want.size(),
                                    " {\"sort_every\": %d, \"tile\": [%d, %d, %d], \"halo\": %d, \"order\": %d}",
                                    &t.sort_every, &t.tile[0], &t.tile[1], &t.tile[2], &t.halo, &t.order);
        if (got == 6 || got == 5) {
            *out = t;
            st = PIC_OK;
        }
    }
    std::fclose(f);
    return st;
}

extern "C" pic_status pic_tune_cache_store(const char* path, const char* key, const pic_tuning* t)
{
    if (!path || !key || !t || std::strchr(key, '"') || std::strchr(key, '\n')) return PIC_EINVAL;
    std::vector<std::string> keep;
    const std::string mine = std::string("\"") + key + "\":";
    if (std::FILE* f = std::fopen(path, "r")) {
        char line[1024];
        while (std::fgets(line, sizeof line, f)) {
            std::string l(line);
            while (!l.empty() && (l.back() == '\n' || l.back() == ',' || l.back() == '\r')) l.pop_back();
            if (l.size() < 2 || l[0] != '"' || l.compare(0, mine.size(), mine) == 0) continue;
            keep.push_back(l);
        }
        std::fclose(f);
    }
    char buf[512];
    std::snprintf(buf, sizeof buf, "%s {\"sort_every\": %d, \"tile\": [%d, %d, %d], \"halo\": %d, \"order\": %d}",
                  mine.c_str(), t->sort_every, t->tile[0], t->tile[1], t->tile[2], t->halo, t->order);
    keep.push_back(buf);
    const std::string tmp = std::string(path) + ".tmp";
    std::FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return PIC_EINVAL;
    std::fputs("{\n", f);
    for (size_t i = 0; i < keep.size(); ++i) std::fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    std::fputs("}\n", f);
    const bool ok = std::fclose(f) == 0 && std::rename(tmp.c_str(), path) == 0;
    return ok ? PIC_OK : PIC_EINVAL;
}
