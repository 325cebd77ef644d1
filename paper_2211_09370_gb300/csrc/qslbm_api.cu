// qslbm C ABI: parameter mapping, wall markers and IB weights, device memory,
// CUDA-graph stepping, diagnostics and state transfer.  See include/qslbm.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qslbm.h"
#include "qslbm_internal.h"

using qslbm::State;

// NVTX range over a host-side phase (shown by profilers that record NVTX; a
// no-op otherwise): "qslbm step", "magnetic sweeps + IB on b", "force + flow +
// IB on u", "diagnostics", "state transfer".
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct qslbm_handle {
    State s;
};

namespace {

thread_local std::string g_last_error;

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return QSLBM_ECUDA;
}

#define QCHK(call)                                      \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

const qslbm::Ops& ops(const State& s) {
    return s.p.precision == QSLBM_FP64 ? qslbm::ops_f64() : qslbm::ops_f32();
}

int dev_alloc(State& s, void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cuda_fail(e, "cudaMalloc");
        return e == cudaErrorMemoryAllocation ? QSLBM_ENOMEM : QSLBM_ECUDA;
    }
    s.allocations.push_back(*p);
    s.device_bytes += (long long)bytes;
    return QSLBM_OK;
}

template <typename V>
int upload(State& s, void** dst, const std::vector<V>& v) {
    size_t bytes = std::max<size_t>(1, v.size()) * sizeof(V);
    int rc = dev_alloc(s, dst, bytes);
    if (rc) return rc;
    if (!v.empty()) QCHK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return QSLBM_OK;
}

// Upload a binary64 host vector in the handle's storage precision.
int upload_real(State& s, void** dst, const std::vector<double>& v) {
    if (s.p.precision == QSLBM_FP64) return upload(s, dst, v);
    std::vector<float> f(v.begin(), v.end());
    return upload(s, dst, f);
}

// N_mag = ceil(c) with c = 2 eta / c_m^2 (Sec. V.G); a c within a relative
// 1e-12 of an integer counts as that integer.
int ceil_rel(double v) {
    double r = std::nearbyint(v);
    if (std::fabs(v - r) <= 1e-12 * std::fabs(v)) return (int)r;
    return (int)std::ceil(v);
}

// Map the problem statement to lattice units.  L = D/2 (Sec. II groups with the
// pipe radius as length, Sec. IV); U0 rule: Mach, tau <= 1 and an explicit
// Lorentz drag B0^2/eta <= 1/2 per step.
int map_units(const qslbm_params& p, qslbm_units& u) {
    std::memset(&u, 0, sizeof(u));
    u.cs2 = 1.0 / 3.0;
    u.cm2 = p.dim == 2 ? 1.0 / 3.0 : 1.0 / 4.0;
    u.R = 0.5 * p.diameter;
    double U0 = p.U0;
    if (!(U0 > 0)) {
        U0 = 0.05;
        if (p.flow_scheme != QSLBM_FLOW_MACROSCOPIC) U0 = std::min(U0, p.Re * u.cs2 / (2.0 * u.R));
        if (p.Ha > 0) U0 = std::min(U0, p.Re * u.R / (2.0 * p.Ha * p.Ha));
    }
    u.U0 = U0;
    u.nu = U0 * u.R / p.Re;
    // time step dt/gamma (Sec. VII); the macroscopic scheme's c = 6 nu (Sec. V.G)
    const double g = p.flow_scheme == QSLBM_FLOW_MACROSCOPIC ? 6.0 * u.nu : (p.gamma > 0 ? p.gamma : 1.0);
    u.gamma = g;
    u.tau = p.flow_scheme == QSLBM_FLOW_MACROSCOPIC ? 1.0 : u.nu / (g * u.cs2) + 0.5;
    u.eta = U0 * u.R / p.Rm;
    u.B0 = p.Ha * std::sqrt(u.eta * u.nu) / u.R;
    u.F0 = (p.geometry == QSLBM_CHANNEL ? 2.0 : 4.0) * u.nu * U0 / (u.R * u.R);
    u.c_mag = 2.0 * u.eta / (g * u.cm2);
    u.tau_m = 1.0;
    u.flow_q = p.dim == 2 ? 9 : (p.flow_q == 27 ? 27 : 19);
    int n = p.n_mag > 0 ? p.n_mag : ceil_rel(u.c_mag);
    if (p.n_mag <= 0 && p.n_mag_cap > 0) n = std::min(n, p.n_mag_cap);
    u.n_mag = std::max(n, 1);
    if (p.mag_scheme == QSLBM_MAG_TIME) {
        // the field lattice at the flow's speed: eta = c_m^2 (tau_m - 1/2)
        u.c_mag = 1.0;
        u.tau_m = u.eta / (g * u.cm2) + 0.5;
        u.n_mag = 1;
    }
    double nu_ref = p.nu_ref > 0 ? p.nu_ref : u.nu / g;
    // eta_ref: c_m^2/2 for the tau_m = 1 sweeps (lambda_m = c); the per-step
    // eta for the time-resolved update (lambda_m = 1: below one the scaling's
    // pole at d = 1/(1 - lambda_m) falls inside the rings' range of d)
    double eta_ref = p.eta_ref > 0 ? p.eta_ref : (p.mag_scheme == QSLBM_MAG_TIME ? u.eta / g : 0.5 * u.cm2);
    u.lambda = u.nu / g / nu_ref;
    u.lambda_m = u.eta / g / eta_ref;
    return QSLBM_OK;
}

// Refusal of a parameter set, with its reason left in qslbm_last_error.
int refuse(const std::string& why) {
    g_last_error = "invalid parameters: " + why;
    return QSLBM_EINVAL;
}

int validate(const qslbm_params& p) {
    if (p.dim != 2 && p.dim != 3) return refuse("dim must be 2 or 3");
    if (p.nx < 1 || p.ny < 1 || p.nz < 1) return refuse("nx, ny and nz must be at least 1");
    if (p.dim == 2 && p.nz != 1) return refuse("a 2-D domain has nz = 1");
    if (p.geometry < QSLBM_CHANNEL || p.geometry > QSLBM_PERIODIC) return refuse("unknown geometry");
    if (!(p.diameter > 0)) return refuse("diameter must be positive");
    if (!(p.Re > 0) || !(p.Rm > 0)) return refuse("Re and Rm must be positive");
    if (!(p.Ha >= 0)) return refuse("Ha must not be negative");
    if (!(p.marker_spacing > 0)) return refuse("marker_spacing must be positive");
    if (p.b0_kind != QSLBM_B0_UNIFORM && p.b0_kind != QSLBM_B0_TANH && p.b0_kind != QSLBM_B0_FIELD)
        return refuse("unknown b0_kind");
    if (p.b0_kind == QSLBM_B0_FIELD && !p.b0_field) return refuse("b0_kind = field needs b0_field");
    if (p.b0_kind == QSLBM_B0_TANH && !(p.ramp_width > 0)) return refuse("ramp_width must be positive");
    if (p.force_amp != 0.0 && !(p.force_period > 0)) return refuse("a pulsating force needs force_period > 0");
    if (p.precision != QSLBM_FP32 && p.precision != QSLBM_FP64) return refuse("unknown precision");
    if (p.n_mag < 0 || p.perturb < 0 || p.nu_ref < 0 || p.eta_ref < 0)
        return refuse("n_mag, perturb, nu_ref and eta_ref must not be negative");
    if (p.sweep_kernel < QSLBM_SWEEP_AUTO || p.sweep_kernel > QSLBM_SWEEP_FUSED) return refuse("unknown sweep_kernel");
    if (p.init_kind != QSLBM_INIT_REST && p.init_kind != QSLBM_INIT_POISEUILLE) return refuse("unknown init_kind");
    if (p.dim == 3 && p.flow_q != 0 && p.flow_q != 19 && p.flow_q != 27) return refuse("3-D flow_q is 19 or 27");
    if (p.dim == 2 && p.flow_q != 0 && p.flow_q != 9) return refuse("2-D flow_q is 9");
    if (p.flow_scheme != QSLBM_FLOW_SINGLE_STEP && p.flow_scheme != QSLBM_FLOW_MACROSCOPIC)
        return refuse("unknown flow_scheme");
    if (p.flow_scheme == QSLBM_FLOW_MACROSCOPIC) {
        if (!(p.gamma == 0.0 || p.gamma == 1.0))  // the scheme sets the time step
            return refuse("the macroscopic flow scheme sets gamma itself");
        qslbm_units u;
        map_units(p, u);
        if (!(6.0 * u.nu >= 1.0 - 1e-12))
            return refuse("macroscopic flow scheme: 6 nu = " + std::to_string(6.0 * u.nu) + " < 1 (tau < 1)");
    }
    {
        // accelerated sweep: the checkerboard gain (2 w_0 - 2 + alpha)/alpha
        // stays >= -1 only for alpha >= 1 - w_0 (w_0 = 1/4 on D3Q7, 1/3 on D2Q5)
        const double a = p.alpha == 0.0 ? 1.0 : p.alpha;
        const double w0 = p.dim == 3 ? 0.25 : 1.0 / 3.0;
        if (!(a >= 1.0 - w0 - 1e-12 && a <= 1.0))
            return refuse("alpha outside [" + std::to_string(1.0 - w0) + ", 1], the sweep's stable range");
        if (p.mag_scheme != QSLBM_MAG_QS && p.mag_scheme != QSLBM_MAG_TIME) return refuse("unknown mag_scheme");
        if (p.mag_scheme == QSLBM_MAG_TIME && a != 1.0)
            return refuse("the time-resolved magnetic update takes no alpha");
        if (!(p.gamma >= 0.0) || p.gamma > 1e6) return refuse("gamma outside [0, 1e6]");
    }
    if (p.mag_scheme == QSLBM_MAG_TIME) {
        // checkerboard gain (2 tau_m - 1)(2 w_0 - 1) - 2 (tau_m - 1) >= -1
        qslbm_units u;
        map_units(p, u);
        const double tmax = p.dim == 3 ? 7.0 / 6.0 : 5.0 / 4.0;
        if (!(u.tau_m > 0.5 && u.tau_m <= tmax + 1e-12))
            return refuse("time-resolved magnetic update: tau_m = " + std::to_string(u.tau_m) + " outside (1/2, " +
                          std::to_string(tmax) + "]");
    }
    // kernels index the three components of a field with 32-bit offsets
    long long n = (long long)p.nx * p.ny * p.nz;
    if (3 * n > (1LL << 31) - 1) return refuse("more than (2^31 - 1)/3 nodes");
    return QSLBM_OK;
}

// Base node and 1-D weights of the Lagrange kernel (Sec. V.B) for coordinate
// X: n0 is the node with n0 - X in (-1/2, 1/2]; the weights of n0 - 1, n0,
// n0 + 1 are r(r+1)/2, 1 - r^2, r(r-1)/2 with r = n0 - X.
void kernel_weights(double X, int& n0, double w[3]) {
    long long k = (long long)std::floor(X + 0.5);
    double r = (double)k - X;
    if (r > 0.5) {
        --k;
        r = (double)k - X;
    } else if (r <= -0.5) {
        ++k;
        r = (double)k - X;
    }
    n0 = (int)k;
    w[0] = 0.5 * r * (r + 1.0);
    w[1] = 1.0 - r * r;
    w[2] = 0.5 * r * (r - 1.0);
}

int wrapn(long long i, int n) {
    long long r = i % n;
    return (int)(r < 0 ? r + n : r);
}

// Markers: channel walls y = cy -/+ D/2 with one marker per spacing along x on
// every z plane; pipe rings of round(pi D / spacing) markers at every integer
// z (Sec. V.B, Fig. 3).  Then W = sum_j D(. - X_j), d_j = sum_k D(x_k - X_j)
// W(x_k) (Sec. V.C), s_j and s^m_j (Sec. V.E, V.F), and the shell CSR.
int build_markers(State& s) {
    qslbm::HostIB& h = s.hib;
    const qslbm_params& p = s.p;
    const int planes = s.nz;
    h.ring_off.assign(planes + 1, 0);
    if (p.geometry == QSLBM_CHANNEL) {
        long long per = std::llround(p.nx / p.marker_spacing);
        for (int z = 0; z < planes; ++z) {
            for (int w = 0; w < 2; ++w)
                for (long long i = 0; i < per; ++i) {
                    h.X.push_back((double)i * p.marker_spacing);
                    h.Y.push_back(w == 0 ? s.cy - s.R : s.cy + s.R);
                    h.zplane.push_back(z);
                }
            h.ring_off[z + 1] = (int)h.X.size();
        }
    } else if (p.geometry == QSLBM_PIPE) {
        long long nth = std::llround(M_PI * p.diameter / p.marker_spacing);
        if (nth < 3) {
            g_last_error = "invalid parameters: a pipe ring needs at least 3 markers (pi D / marker_spacing)";
            return QSLBM_EINVAL;
        }
        for (int z = 0; z < planes; ++z) {
            for (long long i = 0; i < nth; ++i) {
                double th = 2.0 * M_PI * (double)i / (double)nth;
                h.X.push_back(s.cx + s.R * std::cos(th));
                h.Y.push_back(s.cy + s.R * std::sin(th));
                h.zplane.push_back(z);
            }
            h.ring_off[z + 1] = (int)h.X.size();
        }
    } else {
        for (int z = 0; z < planes; ++z) h.ring_off[z + 1] = 0;
    }
    const int nm = (int)h.X.size();
    h.ix.resize(3 * nm);
    h.iy.resize(3 * nm);
    h.wx.resize(3 * nm);
    h.wy.resize(3 * nm);
    for (int j = 0; j < nm; ++j) {
        int x0, y0;
        kernel_weights(h.X[j], x0, &h.wx[3 * j]);
        kernel_weights(h.Y[j], y0, &h.wy[3 * j]);
        for (int a = 0; a < 3; ++a) {
            h.ix[3 * j + a] = wrapn((long long)x0 - 1 + a, s.nx);
            h.iy[3 * j + a] = wrapn((long long)y0 - 1 + a, s.ny);
        }
    }
    h.max_ring = 0;
    for (int z = 0; z < planes; ++z) h.max_ring = std::max(h.max_ring, h.ring_off[z + 1] - h.ring_off[z]);
    if ((size_t)3 * h.max_ring * (p.precision == QSLBM_FP64 ? 8 : 4) > 48 * 1024) {
        // the per-plane IB kernels keep a plane's marker deltas in shared memory
        g_last_error = "wall ring of " + std::to_string(h.max_ring) + " markers per plane exceeds the limit of " +
                       std::to_string(48 * 1024 / (3 * (p.precision == QSLBM_FP64 ? 8 : 4))) + " for this precision";
        return QSLBM_EINVAL;
    }
    // d_j and the scalings
    const long long P = (long long)s.nx * s.ny;
    std::vector<double> W;
    h.shell_off.assign(planes + 1, 0);
    h.d.assign(nm, 0.0);
    h.s.assign(nm, 0.0);
    h.sm.assign(nm, 0.0);
    for (int z = 0; z < planes; ++z) {
        const int m0 = h.ring_off[z], m1 = h.ring_off[z + 1];
        h.shell_off[z] = (int)h.shell_xy.size();
        h.shell_off[z + 1] = (int)h.shell_xy.size();
        if (m0 == m1) continue;
        W.assign(P, 0.0);
        for (int j = m0; j < m1; ++j)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) W[(long long)h.iy[3 * j + b] * s.nx + h.ix[3 * j + a]] += h.wx[3 * j + a] * h.wy[3 * j + b];
        for (int j = m0; j < m1; ++j) {
            double acc = 0.0;
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a)
                    acc += h.wx[3 * j + a] * h.wy[3 * j + b] * W[(long long)h.iy[3 * j + b] * s.nx + h.ix[3 * j + a]];
            h.d[j] = acc;
            const double l = s.units.lambda, lm = s.units.lambda_m;
            h.s[j] = l / (acc * (1.0 + acc * (l - 1.0)));
            h.sm[j] = lm / (acc * (1.0 + acc * (lm - 1.0)));
        }
        // shell CSR of plane z: nodes with a nonzero weight, markers in ring order
        struct Ent {
            int xy, l;
            double w;
        };
        std::vector<Ent> ents;
        for (int j = m0; j < m1; ++j)
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    double w = h.wx[3 * j + a] * h.wy[3 * j + b];
                    if (w != 0.0) ents.push_back({h.iy[3 * j + b] * s.nx + h.ix[3 * j + a], j - m0, w});
                }
        std::stable_sort(ents.begin(), ents.end(), [](const Ent& x, const Ent& y) { return x.xy < y.xy; });
        for (size_t e = 0; e < ents.size(); ++e) {
            if (e == 0 || ents[e].xy != ents[e - 1].xy) {
                h.shell_xy.push_back(ents[e].xy);
                h.csr_off.push_back((int)h.csr_m.size());
            }
            h.csr_m.push_back(ents[e].l);
            h.csr_w.push_back(ents[e].w);
        }
        h.shell_off[z + 1] = (int)h.shell_xy.size();
    }
    h.csr_off.push_back((int)h.csr_m.size());
    h.max_shell = 0;
    h.max_nnz = 0;
    for (int z = 0; z < planes; ++z) {
        const int ns = h.shell_off[z + 1] - h.shell_off[z];
        h.max_shell = std::max(h.max_shell, ns);
        if (ns > 0)
            h.max_nnz = std::max(h.max_nnz, h.csr_off[h.shell_off[z + 1]] - h.csr_off[h.shell_off[z]]);
    }
    for (double v : h.d)
        if (!(v > 0)) {
            g_last_error = "invalid parameters: a marker has no lattice node in its support (d_j = 0)";
            return QSLBM_EINVAL;
        }
    return QSLBM_OK;
}

// True when every z plane's ring and shell tables (in-plane indices, weights,
// scalings, CSR) equal plane 0's, as for a straight pipe with a ring on every
// plane; per-plane IB kernels then read one plane's tables for all planes.
bool ib_tables_z_invariant(const State& s, const std::vector<int>& q9, const std::vector<double>& w9) {
    const qslbm::HostIB& h = s.hib;
    if (s.nz <= 1) return true;
    const int R = h.ring_off[1] - h.ring_off[0];
    const int S = h.shell_off[1] - h.shell_off[0];
    for (int z = 1; z < s.nz; ++z) {
        const int m0 = h.ring_off[z], s0 = h.shell_off[z];
        if (h.ring_off[z + 1] - m0 != R || h.shell_off[z + 1] - s0 != S) return false;
        for (int j = 0; j < R; ++j) {
            if (h.s[m0 + j] != h.s[j] || h.sm[m0 + j] != h.sm[j]) return false;
            for (int k = 0; k < 9; ++k)
                if (q9[9 * (m0 + j) + k] != q9[9 * j + k] || w9[9 * (m0 + j) + k] != w9[9 * j + k]) return false;
        }
        for (int i = 0; i < S; ++i) {
            if (h.shell_xy[s0 + i] != h.shell_xy[i]) return false;
            const int e0 = h.csr_off[s0 + i], e1 = h.csr_off[s0 + i + 1];
            if (e1 - e0 != h.csr_off[i + 1] - h.csr_off[i]) return false;
            for (int e = 0; e < e1 - e0; ++e)
                if (h.csr_m[e0 + e] != h.csr_m[h.csr_off[i] + e] || h.csr_w[e0 + e] != h.csr_w[h.csr_off[i] + e])
                    return false;
        }
    }
    return true;
}

int upload_ib(State& s) {
    qslbm::HostIB& h = s.hib;
    qslbm::DeviceIB& d = s.ib;
    int rc;
    // per marker the nine in-plane node indices and weights D = D_x D_y
    const size_t nm = h.X.size();
    std::vector<int> q9(9 * nm);
    std::vector<double> w9(9 * nm);
    for (size_t j = 0; j < nm; ++j)
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                q9[9 * j + 3 * b + a] = h.iy[3 * j + b] * s.nx + h.ix[3 * j + a];
                w9[9 * j + 3 * b + a] = h.wx[3 * j + a] * h.wy[3 * j + b];
            }
    {
        // position of each support node in its plane's shell list (sorted by
        // in-plane index); zero-weight support nodes point at entry 0
        std::vector<int> slot(9 * nm, 0);
        for (int z = 0; z < s.nz; ++z) {
            const int* sb = h.shell_xy.data() + h.shell_off[z];
            const int S = h.shell_off[z + 1] - h.shell_off[z];
            for (int j = h.ring_off[z]; j < h.ring_off[z + 1]; ++j)
                for (int k = 0; k < 9; ++k) {
                    if (w9[9 * j + k] == 0.0) continue;
                    const int* it = std::lower_bound(sb, sb + S, q9[9 * j + k]);
                    if (it == sb + S || *it != q9[9 * j + k]) return QSLBM_EINVAL;  // not reachable
                    slot[9 * j + k] = (int)(it - sb);
                }
        }
        if ((rc = upload(s, (void**)&d.mk_slot, slot))) return rc;
    }
    if ((rc = upload(s, (void**)&d.ring_off, h.ring_off))) return rc;
    if ((rc = upload(s, (void**)&d.mk_q, q9))) return rc;
    if ((rc = upload_real(s, &d.mk_w, w9))) return rc;
    if ((rc = upload_real(s, &d.mk_s, h.s))) return rc;
    if ((rc = upload_real(s, &d.mk_sm, h.sm))) return rc;
    {
        const long long P = (long long)s.nx * s.ny;
        std::vector<int> mbase(nm), snode(h.shell_xy.size()), cmg(h.csr_m.size());
        for (size_t j = 0; j < nm; ++j) mbase[j] = (int)(h.zplane[j] * P);
        for (int z = 0; z < s.nz; ++z)
            for (int i = h.shell_off[z]; i < h.shell_off[z + 1]; ++i) {
                snode[i] = (int)(z * P + h.shell_xy[i]);
                for (int e = h.csr_off[i]; e < h.csr_off[i + 1]; ++e) cmg[e] = h.ring_off[z] + h.csr_m[e];
            }
        if ((rc = upload(s, (void**)&d.mk_base, mbase))) return rc;
        if ((rc = upload(s, (void**)&d.shell_node, snode))) return rc;
        if ((rc = upload(s, (void**)&d.csr_mg, cmg))) return rc;
        if ((rc = dev_alloc(s, &d.delta, (size_t)3 * std::max<size_t>(1, nm) * s.esz))) return rc;
    }
    if ((rc = upload(s, (void**)&d.shell_off, h.shell_off))) return rc;
    if ((rc = upload(s, (void**)&d.shell_xy, h.shell_xy))) return rc;
    if ((rc = upload(s, (void**)&d.csr_off, h.csr_off))) return rc;
    if ((rc = upload(s, (void**)&d.csr_m, h.csr_m))) return rc;
    if ((rc = upload_real(s, &d.csr_w, h.csr_w))) return rc;
    d.nm = (int)h.X.size();
    d.ns = (int)h.shell_xy.size();
    d.nnz = (int)h.csr_m.size();
    d.max_ring = h.max_ring;
    d.max_shell = h.max_shell;
    d.max_nnz = h.max_nnz;
    d.zinv = ib_tables_z_invariant(s, q9, w9) ? 1 : 0;
    {
        // each shell node's markers and weights in CSR order, padded to a
        // multiple of four entries (plane 0's nodes alone when every plane
        // carries plane 0's tables)
        const int nsp = d.zinv ? h.shell_off[1] : (int)h.shell_xy.size();
        int kmax = 0;
        for (int i = 0; i < nsp; ++i) kmax = std::max(kmax, h.csr_off[i + 1] - h.csr_off[i]);
        const int K = (kmax + 3) / 4 * 4;
        d.pad_k = 0;
        if (K > 0 && K <= qslbm::kMaxPadK) {
            std::vector<int> pm((size_t)nsp * K, 0);
            std::vector<double> pw((size_t)nsp * K, 0.0);
            for (int i = 0; i < nsp; ++i)
                for (int e = h.csr_off[i]; e < h.csr_off[i + 1]; ++e) {
                    pm[(size_t)i * K + (e - h.csr_off[i])] = h.csr_m[e];
                    pw[(size_t)i * K + (e - h.csr_off[i])] = h.csr_w[e];
                }
            if ((rc = upload(s, (void**)&d.pad_m, pm))) return rc;
            if ((rc = upload_real(s, &d.pad_w, pw))) return rc;
            d.pad_k = K;
        }
    }
    return QSLBM_OK;
}

// The fused sweep + IB kernel (FP32): rows per band TY, the per-band IB
// tables (plane 0's ring: every plane carries it) and the tensor maps of b
// and u.  Leaves s.fused false when the kernel does not apply: other
// precision or dimension, nx not a multiple of 4 or above 256, planes with
// different rings, no band height that fits shared memory and keeps every
// 3-row box off the periodic boundary.
int plan_fused(State& s) {
    s.fused = false;
    if (s.p.precision != QSLBM_FP32 || s.dim != 3) return QSLBM_OK;
    if (s.nx % 4 != 0 || s.nx > 256 || s.ny < 8 || s.nz < 3) return QSLBM_OK;
    if (s.ib.nm > 0 && !s.ib.zinv) return QSLBM_OK;
    if (3LL * s.n >= (1LL << 31)) return QSLBM_OK;
    int dev = 0, optin = 0;
    QCHK(cudaGetDevice(&dev));
    QCHK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const qslbm::HostIB& h = s.hib;
    const int R0 = h.ring_off.size() > 1 ? h.ring_off[1] - h.ring_off[0] : 0;
    const int S0 = h.shell_off.size() > 1 ? h.shell_off[1] - h.shell_off[0] : 0;
    const int ny = s.ny, nx = s.nx;
    // tallest band whose swept rows give at most one node pair per thread
    int TY = std::min(ny - 6, qslbm::kFusedMaxThreads * 2 / nx - 4);
    for (; TY >= 3; --TY) {
        const int bands = (ny + TY - 1) / TY;
        if (bands < 2) continue;
        // every 3-row box lies on one side of the periodic boundary
        bool ok = true;
        for (int b = 0; b < bands && ok; ++b) {
            const int y0 = std::min(b * TY, ny - TY);
            if (y0 > 0 && y0 < 3) ok = false;
            if (y0 + TY != ny && y0 + TY + 3 > ny) ok = false;
        }
        if (!ok) continue;
        // local row of y in band b's swept rows (y0 - 2 .. y0 + TY + 1), or -1
        auto local = [&](int y0, int y) {
            const int r = ((y - (y0 - 2)) % ny + ny) % ny;
            return r < TY + 4 ? r : -1;
        };
        // markers of each band: support centred on rows y0 - 1 .. y0 + TY
        std::vector<std::vector<int>> mk(bands), sh(bands);
        for (int b = 0; b < bands; ++b) {
            const int y0 = std::min(b * TY, ny - TY);
            for (int j = 0; j < R0; ++j) {
                const int r = local(y0, h.iy[3 * j + 1]);
                if (r >= 1 && r <= TY + 2) mk[b].push_back(j);
            }
            for (int i = 0; i < S0; ++i) {
                const int y = h.shell_xy[i] / nx;
                if (y >= y0 && y < y0 + TY) sh[b].push_back(i);
            }
        }
        int Mmax = 1, Smax = 1, K = 4;
        for (int b = 0; b < bands; ++b) {
            Mmax = std::max(Mmax, (int)mk[b].size());
            Smax = std::max(Smax, (int)sh[b].size());
        }
        Mmax = (Mmax + 3) / 4 * 4;  // 16-byte alignment of the tables in shared memory
        Smax = (Smax + 3) / 4 * 4;
        for (int i = 0; i < S0; ++i) K = std::max(K, (h.csr_off[i + 1] - h.csr_off[i] + 3) / 4 * 4);
        int slots = 5;
        size_t smem = qslbm::fused_smem_bytes(nx, TY, Mmax, Smax, K, slots);
        if (smem + 1024 > (size_t)optin) smem = qslbm::fused_smem_bytes(nx, TY, Mmax, Smax, K, slots = 4);
        if (smem + 1024 > (size_t)optin) continue;
        std::vector<int> mk_cnt(bands), mk_off((size_t)bands * Mmax * 9, 0), sh_cnt(bands),
            sh_off((size_t)bands * Smax, 0), sh_m((size_t)bands * Smax * K, 0), sh_ce((size_t)bands * Smax, 0);
        std::vector<double> mk_w((size_t)bands * Mmax * 9, 0.0), mk_s((size_t)bands * Mmax, 0.0),
            sh_w((size_t)bands * Smax * K, 0.0);
        for (int b = 0; b < bands; ++b) {
            const int y0 = std::min(b * TY, ny - TY);
            std::vector<int> pos(R0, -1);  // marker -> index in the band's list
            mk_cnt[b] = (int)mk[b].size();
            for (int m = 0; m < mk_cnt[b]; ++m) {
                const int j = mk[b][m];
                pos[j] = m;
                const size_t e = ((size_t)b * Mmax + m) * 9;
                for (int bb = 0; bb < 3; ++bb)
                    for (int a = 0; a < 3; ++a) {
                        const int r = local(y0, h.iy[3 * j + bb]);
                        if (r < 0) return QSLBM_EINVAL;  // not reachable: the support is within one row
                        mk_off[e + 3 * bb + a] = r * nx + h.ix[3 * j + a];
                        mk_w[e + 3 * bb + a] = h.wx[3 * j + a] * h.wy[3 * j + bb];
                    }
                mk_s[(size_t)b * Mmax + m] = h.sm[j];
            }
            sh_cnt[b] = (int)sh[b].size();
            for (int k = 0; k < sh_cnt[b]; ++k) {
                const int i = sh[b][k];
                const int y = h.shell_xy[i] / nx, x = h.shell_xy[i] - y * nx;
                sh_off[(size_t)b * Smax + k] = (y - y0 + 2) * nx + x;
                sh_ce[(size_t)b * Smax + k] = h.csr_off[i + 1] - h.csr_off[i];
                for (int e = h.csr_off[i]; e < h.csr_off[i + 1]; ++e) {
                    const int m = pos[h.csr_m[e]];
                    if (m < 0) return QSLBM_EINVAL;  // not reachable: its markers are the band's
                    const size_t q = ((size_t)b * Smax + k) * K + (e - h.csr_off[i]);
                    sh_m[q] = m;
                    sh_w[q] = h.csr_w[e];
                }
            }
        }
        int rc;
        if ((rc = upload(s, (void**)&s.fu_mk_cnt, mk_cnt))) return rc;
        if ((rc = upload(s, (void**)&s.fu_mk_off, mk_off))) return rc;
        if ((rc = upload_real(s, (void**)&s.fu_mk_w, mk_w))) return rc;
        if ((rc = upload_real(s, (void**)&s.fu_mk_s, mk_s))) return rc;
        if ((rc = upload(s, (void**)&s.fu_sh_cnt, sh_cnt))) return rc;
        if ((rc = upload(s, (void**)&s.fu_sh_off, sh_off))) return rc;
        if ((rc = upload(s, (void**)&s.fu_sh_m, sh_m))) return rc;
        if ((rc = upload_real(s, (void**)&s.fu_sh_w, sh_w))) return rc;
        if ((rc = upload(s, (void**)&s.fu_sh_ce, sh_ce))) return rc;
        if ((rc = dev_alloc(s, (void**)&s.fu_err, sizeof(int)))) return rc;
        QCHK(cudaMemsetAsync(s.fu_err, 0, sizeof(int), s.stream));
        // tensor maps: b[i] and u[i] as 4-D (x, y, z, component) FP32 tensors,
        // boxes of 3 rows and of TY rows of one component
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        QCHK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) {
            g_last_error = "cuTensorMapEncodeTiled is not available";
            return QSLBM_ECUDA;
        }
        auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)s.nz, 3};
        const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)s.n * 4};
        const cuuint32_t box3[4] = {(cuuint32_t)nx, 3, 1, 1};
        const cuuint32_t boxt[4] = {(cuuint32_t)nx, (cuuint32_t)TY, 1, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        for (int i = 0; i < 2; ++i) {
            CUtensorMap* maps[4] = {&s.fu_map_b3[i], &s.fu_map_bt[i], &s.fu_map_u3[i], &s.fu_map_ut[i]};
            void* ptrs[4] = {s.b[i], s.b[i], s.u[i], s.u[i]};
            for (int f = 0; f < 4; ++f) {
                CUresult r = encode(maps[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, ptrs[f], dims, strides,
                                    f % 2 ? boxt : box3, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) {
                    g_last_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
                    return QSLBM_ECUDA;
                }
            }
        }
        s.fu_TY = TY;
        s.fu_bands = bands;
        s.fu_Mmax = Mmax;
        s.fu_Smax = Smax;
        s.fu_K = K;
        s.fu_smem = smem;
        s.fu_slots = slots;
        s.fused = true;
        QCHK(ops(s).plan_fused(s));
        return QSLBM_OK;
    }
    return QSLBM_OK;
}

// A fused sweep whose copy wait timed out leaves 1 in fu_err; report it once.
int check_fused(State& s) {
    if (!s.fu_err) return QSLBM_OK;
    int err = 0;
    QCHK(cudaMemcpyAsync(&err, s.fu_err, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    if (!err) return QSLBM_OK;
    QCHK(cudaMemsetAsync(s.fu_err, 0, sizeof(int), s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    g_last_error = "fused sweep kernel: a plane copy did not complete in time";
    return QSLBM_ETIMEOUT;
}

double body_force(const State& s, long long t) {
    double f = s.units.F0;
    if (s.p.force_amp != 0.0) f *= 1.0 + s.p.force_amp * std::sin(s.omega * (double)t);
    return f;
}

void release(State& s) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (s.graph[a][b]) cudaGraphExecDestroy(s.graph[a][b]);
    for (void* p : s.allocations) cudaFree(p);
    s.allocations.clear();
    if (s.own_stream && s.stream) cudaStreamDestroy(s.stream);
    s.stream = nullptr;
}

int check_device() {
    int dev = 0;
    QCHK(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    QCHK(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3)) {
        g_last_error = std::string("device is sm_") + std::to_string(prop.major) + std::to_string(prop.minor) +
                       ", the library is built for sm_103a only";
        return QSLBM_EARCH;
    }
    return QSLBM_OK;
}

int create_impl(const qslbm_params* pin, qslbm_handle** out) {
    if (!pin || !out) {
        g_last_error = "qslbm_create: the parameter or output pointer is NULL";
        return QSLBM_EINVAL;
    }
    *out = nullptr;
    int rc = validate(*pin);
    if (rc) return rc;
    if ((rc = check_device())) return rc;
    qslbm_handle* h = new (std::nothrow) qslbm_handle();
    if (!h) return QSLBM_ENOMEM;
    State& s = h->s;
    bool tune_sweep = false;  // AUTO on a domain both FP32 sweep paths take: time them
    s.p = *pin;
    s.dim = s.p.dim;
    s.nx = s.p.nx;
    s.ny = s.p.ny;
    s.nz = s.p.dim == 2 ? 1 : s.p.nz;
    s.n = (long long)s.nx * s.ny * s.nz;
    s.esz = s.p.precision == QSLBM_FP64 ? 8 : 4;
    map_units(s.p, s.units);
    s.units.nodes = s.n;
    s.cx = std::isnan(s.p.center[0]) ? 0.5 * (s.nx - 1) : s.p.center[0];
    s.cy = std::isnan(s.p.center[1]) ? 0.5 * (s.ny - 1) : s.p.center[1];
    s.R = s.units.R;
    s.axis = s.dim == 3 ? 2 : 0;
    s.ig = 1.0 / s.units.gamma;
    // the modulation runs on physical time t/gamma
    s.omega = s.p.force_amp != 0.0 ? 2.0 * M_PI / s.p.force_period * s.ig : 0.0;
    if (s.dim == 3) {
        s.w0 = 0.25;
        s.alpha = s.p.alpha == 0.0 ? 1.0 : s.p.alpha;
        s.w1 = 0.125;
    } else {
        s.w0 = 1.0 / 3.0;
        s.alpha = s.p.alpha == 0.0 ? 1.0 : s.p.alpha;
        s.w1 = 1.0 / 6.0;
    }
    s.kappa = 1.0 / (s.units.c_mag * s.units.cm2);
    for (int a = 0; a < 3; ++a) s.be[a] = s.p.b0_kind == QSLBM_B0_FIELD ? 0.0 : s.units.B0 * s.p.b0_dir[a];
    if ((rc = build_markers(s))) {
        delete h;
        return rc;
    }
    s.units.n_markers = (int)s.hib.X.size();
    s.units.shell_nodes = (long long)s.hib.shell_xy.size();
    if (s.p.stream) {
        s.stream = (cudaStream_t)s.p.stream;
    } else {
        cudaError_t e = cudaStreamCreate(&s.stream);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "cudaStreamCreate");
        }
        s.own_stream = true;
    }
    const size_t fb = (size_t)s.n * s.esz;
    void** fields[] = {&s.drho[0], &s.drho[1]};
    for (void** f : fields)
        if ((rc = dev_alloc(s, f, fb))) goto fail;
    for (int i = 0; i < 2; ++i) {
        if ((rc = dev_alloc(s, &s.u[i], 3 * fb))) goto fail;
        if ((rc = dev_alloc(s, &s.b[i], 3 * fb))) goto fail;
    }
    if ((rc = dev_alloc(s, &s.F, 3 * fb))) goto fail;
    if ((rc = dev_alloc(s, &s.usnap, 3 * fb))) goto fail;
    if ((rc = dev_alloc(s, (void**)&s.tdev, sizeof(long long)))) goto fail;
    s.nblocks_obs = (int)std::min<long long>(1024, (s.n + qslbm::kReduceThreads - 1) / qslbm::kReduceThreads);
    if ((rc = dev_alloc(s, (void**)&s.partial, (size_t)s.nblocks_obs * qslbm::kObs * sizeof(double)))) goto fail;
    if ((rc = dev_alloc(s, (void**)&s.obs_dev, qslbm::kObs * sizeof(double)))) goto fail;
    if (s.p.b0_kind == QSLBM_B0_TANH) {
        s.bext_host.resize(3 * s.nz);
        for (int z = 0; z < s.nz; ++z) {
            double amp = s.units.B0 * 0.5 * (1.0 + std::tanh(((double)z - s.p.ramp_center) / s.p.ramp_width));
            for (int a = 0; a < 3; ++a) s.bext_host[3 * z + a] = amp * s.p.b0_dir[a];
        }
        if ((rc = upload_real(s, &s.bext_z, s.bext_host))) goto fail;
    }
    if (s.p.b0_kind == QSLBM_B0_FIELD) {
        const size_t P = (size_t)s.nx * s.ny;
        std::vector<double> f(3 * P);
        for (size_t i = 0; i < 3 * P; ++i) f[i] = s.units.B0 * s.p.b0_field[i];
        if ((rc = upload_real(s, &s.bext_xy, f))) goto fail;
    }
    s.p.b0_field = nullptr;  // the caller's array is not kept
    if ((rc = upload_ib(s))) goto fail;
    if (s.p.sweep_kernel == QSLBM_SWEEP_AUTO || s.p.sweep_kernel == QSLBM_SWEEP_RESIDENT) {
        cudaError_t e = ops(s).plan_resident(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "plan_resident");
            goto fail;
        }
        if (!s.resident && s.p.sweep_kernel == QSLBM_SWEEP_RESIDENT) {
            g_last_error = "the resident sweep kernel does not fit this domain";
            rc = QSLBM_EINVAL;
            goto fail;
        }
    }
    if (s.resident) {
        const size_t xb = (size_t)2 * 3 * s.n * s.esz;
        const size_t sb = sizeof(unsigned int) * (4 + (size_t)s.nz);
        if ((rc = dev_alloc(s, &s.xbuf, xb))) goto fail;
        if ((rc = dev_alloc(s, &s.rsync, sb))) goto fail;
        cudaError_t e = cudaMemsetAsync(s.rsync, 0, sb, s.stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync");
            goto fail;
        }
    }
    tune_sweep = !s.resident && s.p.sweep_kernel == QSLBM_SWEEP_AUTO;
    if (!s.resident && (s.p.sweep_kernel == QSLBM_SWEEP_AUTO || s.p.sweep_kernel == QSLBM_SWEEP_FUSED)) {
        if ((rc = plan_fused(s))) goto fail;
        if (!s.fused && s.p.sweep_kernel == QSLBM_SWEEP_FUSED) {
            g_last_error = "the fused sweep kernel does not apply to this domain";
            rc = QSLBM_EINVAL;
            goto fail;
        }
        if (s.fused) s.p.sweep_kernel = QSLBM_SWEEP_FUSED;
    }
    if (!s.resident && s.p.sweep_kernel == QSLBM_SWEEP_AUTO) s.p.sweep_kernel = QSLBM_SWEEP_SPLIT;
    {
        cudaError_t e = ops(s).plan_march(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "plan_march");
            goto fail;
        }
    }
    {
        long long zero = 0;
        cudaError_t e = cudaMemcpyAsync(s.tdev, &zero, sizeof(zero), cudaMemcpyHostToDevice, s.stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemcpyAsync");
            goto fail;
        }
        ops(s).init(s, s.stream);
        e = cudaMemcpyAsync(s.usnap, s.u[0], 3 * fb, cudaMemcpyDeviceToDevice, s.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s.stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "init");
            goto fail;
        }
        // initial mass: rho = 1 everywhere
        s.mass0 = (double)s.n;
    }
    if (tune_sweep && s.fused) {
        // both FP32 sweep paths apply: keep the faster on this domain
        cudaError_t e = ops(s).tune_fused(s, &s.units.sweep_us_fused, &s.units.sweep_us_split);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "tune_fused");
            goto fail;
        }
    }
    s.units.sweep_kernel = s.resident ? QSLBM_SWEEP_RESIDENT : s.p.sweep_kernel;
    if (s.fused) {
        s.units.fused_rows = s.fu_TY;
        s.units.fused_bands = s.fu_bands;
        s.units.fused_chunk = s.fu_chunk;
        s.units.fused_ctas = s.fu_bands * s.fu_chunks;
    }
    s.units.device_bytes = s.device_bytes;
    *out = h;
    return QSLBM_OK;
fail:
    release(s);
    delete h;
    return rc;
}

// Steps per captured graph; each graph starts from a given ping-pong parity.
constexpr int kGraphSteps = 1;

int capture_chunk(State& s, int bc, int fc, cudaGraphExec_t* exec) {
    const int save_b = s.bcur, save_f = s.fcur;
    s.bcur = bc;
    s.fcur = fc;
    cudaGraph_t g = nullptr;
    QCHK(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kGraphSteps; ++i) {
        {
            NvtxRange r("magnetic sweeps + IB on b");
            ops(s).sweeps(s, s.units.n_mag, s.stream);
        }
        NvtxRange r("force + flow + IB on u");
        ops(s).force_flow(s, s.stream);
    }
    cudaError_t e = cudaStreamEndCapture(s.stream, &g);
    s.graph_next[bc][fc][0] = s.bcur;
    s.graph_next[bc][fc][1] = s.fcur;
    s.bcur = save_b;
    s.fcur = save_f;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return QSLBM_OK;
}

int step_impl(State& s, long long nsteps) {
    if (nsteps < 0) {
        g_last_error = "negative step count";
        return QSLBM_EINVAL;
    }
    NvtxRange range("qslbm step");
    const qslbm::Ops& o = ops(s);
    long long done = 0;
    while (nsteps - done >= kGraphSteps) {
        cudaGraphExec_t& ex = s.graph[s.bcur][s.fcur];
        if (!ex) {
            int rc = capture_chunk(s, s.bcur, s.fcur, &ex);
            if (rc) return rc;
        }
        QCHK(cudaGraphLaunch(ex, s.stream));
        const int nb = s.graph_next[s.bcur][s.fcur][0], nf = s.graph_next[s.bcur][s.fcur][1];
        s.bcur = nb;
        s.fcur = nf;
        done += kGraphSteps;
    }
    for (; done < nsteps; ++done) {
        {
            NvtxRange r("magnetic sweeps + IB on b");
            o.sweeps(s, s.units.n_mag, s.stream);
        }
        NvtxRange r("force + flow + IB on u");
        o.force_flow(s, s.stream);
    }
    QCHK(cudaGetLastError());
    if (s.launch_error) {
        s.launch_error = false;
        g_last_error = "a launch of the resident or fused sweep kernel failed";
        return QSLBM_ECUDA;
    }
    s.t += nsteps;
    return QSLBM_OK;
}

// A resident launch whose neighbour wait timed out leaves err = 1 in the sync
// block; report it once and reset the counters so the handle stays usable.
int check_resident(State& s) {
    if (!s.resident) return QSLBM_OK;
    int err = 0;
    QCHK(cudaMemcpyAsync(&err, (char*)s.rsync + 2 * sizeof(unsigned int), sizeof(int), cudaMemcpyDeviceToHost,
                         s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    if (!err) return QSLBM_OK;
    QCHK(cudaMemsetAsync(s.rsync, 0, sizeof(unsigned int) * (4 + (size_t)s.nz), s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    g_last_error = "resident sweep kernel: neighbour wait timed out";
    return QSLBM_ETIMEOUT;
}

int ensure_staging(State& s) {
    if (s.staging) return QSLBM_OK;
    return dev_alloc(s, (void**)&s.staging, (size_t)7 * s.n * sizeof(double));
}

int observe_impl(State& s, qslbm_obs* out) {
    NvtxRange range("diagnostics");
    double r[qslbm::kObs];
    ops(s).observe(s, body_force(s, s.t), s.stream);
    QCHK(cudaGetLastError());
    QCHK(cudaMemcpyAsync(r, s.obs_dev, sizeof(r), cudaMemcpyDeviceToHost, s.stream));
    QCHK(cudaMemcpyAsync(s.usnap, s.u[s.fcur], 3 * (size_t)s.n * s.esz, cudaMemcpyDeviceToDevice, s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    if (int rc = check_resident(s)) return rc;
    if (int rc = check_fused(s)) return rc;
    const long long dt = s.t - s.tsnap;
    s.tsnap = s.t;
    if (out) {
        std::memset(out, 0, sizeof(*out));
        const double inv = r[9] > 0 ? 1.0 / r[9] : 0.0;
        out->step = s.t;
        out->mass = r[0];
        out->mass_drift = (r[0] - s.mass0) / s.mass0;
        out->E_k = r[1] * inv;
        out->E_m = r[2] * inv;
        out->pump = r[3] * inv;
        out->visc = -s.units.nu * r[4] * inv;
        out->joule = r[5] * inv;
        out->qs_residual = std::sqrt(r[6] * inv);
        out->steady_residual = (dt > 0 && r[8] > 0) ? std::sqrt(r[7]) / ((double)dt * std::sqrt(r[8])) : 0.0;
        out->nan_flag = r[10] > 0 ? 1 : 0;
    }
    return r[10] > 0 ? QSLBM_EUNSTABLE : QSLBM_OK;
}

int get_fields(State& s, double* rho, double* u, double* b) {
    if (!rho && !u && !b) return QSLBM_OK;
    NvtxRange range("state transfer");
    int rc = ensure_staging(s);
    if (rc) return rc;
    ops(s).to_f64(s, s.stream);
    QCHK(cudaGetLastError());
    const size_t n = (size_t)s.n;
    if (rho) QCHK(cudaMemcpyAsync(rho, s.staging, n * 8, cudaMemcpyDeviceToHost, s.stream));
    if (u) QCHK(cudaMemcpyAsync(u, s.staging + n, 3 * n * 8, cudaMemcpyDeviceToHost, s.stream));
    if (b) QCHK(cudaMemcpyAsync(b, s.staging + 4 * n, 3 * n * 8, cudaMemcpyDeviceToHost, s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    return QSLBM_OK;
}

int set_fields(State& s, const double* rho, const double* u, const double* b, long long t) {
    NvtxRange range("state transfer");
    int rc = ensure_staging(s);
    if (rc) return rc;
    const size_t n = (size_t)s.n;
    int mask = 0;
    if (rho) {
        QCHK(cudaMemcpyAsync(s.staging, rho, n * 8, cudaMemcpyHostToDevice, s.stream));
        mask |= 1;
    }
    if (u) {
        QCHK(cudaMemcpyAsync(s.staging + n, u, 3 * n * 8, cudaMemcpyHostToDevice, s.stream));
        mask |= 2;
    }
    if (b) {
        QCHK(cudaMemcpyAsync(s.staging + 4 * n, b, 3 * n * 8, cudaMemcpyHostToDevice, s.stream));
        mask |= 4;
    }
    if (mask) ops(s).from_f64(s, mask, s.stream);
    QCHK(cudaGetLastError());
    QCHK(cudaMemcpyAsync(s.tdev, &t, sizeof(t), cudaMemcpyHostToDevice, s.stream));
    QCHK(cudaMemcpyAsync(s.usnap, s.u[s.fcur], 3 * n * s.esz, cudaMemcpyDeviceToDevice, s.stream));
    QCHK(cudaStreamSynchronize(s.stream));
    s.t = t;
    s.tsnap = t;
    return QSLBM_OK;
}

}  // namespace

namespace qslbm {
void set_last_error(const std::string& msg) { g_last_error = msg; }
const State& handle_state(const qslbm_handle* h) { return h->s; }
State& handle_state_mut(qslbm_handle* h) { return h->s; }
}  // namespace qslbm

// A NULL handle or an out-of-range argument of an ABI call.
static int bad_argument(const char* what) {
    g_last_error = what;
    return QSLBM_EINVAL;
}

extern "C" {

void qslbm_params_init(qslbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 3;
    p->nx = p->ny = p->nz = 1;
    p->geometry = QSLBM_PIPE;
    p->center[0] = p->center[1] = NAN;
    p->marker_spacing = 1.0;
    p->b0_kind = QSLBM_B0_UNIFORM;
    p->b0_dir[0] = 1.0;
    p->ramp_width = 1.0;
    p->n_mag_cap = 270;
    p->precision = QSLBM_FP32;
    p->alpha = 1.0;
}

int qslbm_create(const qslbm_params* p, qslbm_handle** out) {
    try {
        return create_impl(p, out);
    } catch (...) {
        return QSLBM_ENOMEM;
    }
}

int qslbm_get_units(const qslbm_handle* h, qslbm_units* out) {
    if (!h || !out) return bad_argument("qslbm_get_units: NULL argument");
    *out = h->s.units;
    out->device_bytes = h->s.device_bytes;
    return QSLBM_OK;
}

int qslbm_step(qslbm_handle* h, int64_t nsteps) {
    if (!h) return bad_argument("qslbm_step: NULL handle");
    return step_impl(h->s, nsteps);
}

int qslbm_mag_sweeps(qslbm_handle* h, int32_t nsweeps) {
    if (!h || nsweeps < 0) return bad_argument("qslbm_mag_sweeps: NULL handle or negative sweep count");
    NvtxRange range("magnetic sweeps + IB on b");
    ops(h->s).sweeps(h->s, nsweeps, h->s.stream);
    QCHK(cudaGetLastError());
    if (h->s.launch_error) {
        h->s.launch_error = false;
        g_last_error = "a launch of the resident or fused sweep kernel failed";
        return QSLBM_ECUDA;
    }
    return QSLBM_OK;
}

int qslbm_observables(qslbm_handle* h, qslbm_obs* out, double* rho, double* u, double* b) {
    if (!h) return bad_argument("qslbm_observables: NULL handle");
    int rc = observe_impl(h->s, out);
    if (rc && rc != QSLBM_EUNSTABLE) return rc;
    int rc2 = get_fields(h->s, rho, u, b);
    return rc2 ? rc2 : rc;
}

int qslbm_get_state(qslbm_handle* h, double* rho, double* u, double* b, int64_t* t) {
    if (!h) return bad_argument("qslbm_get_state: NULL handle");
    int rc = get_fields(h->s, rho, u, b);
    if (rc) return rc;
    QCHK(cudaStreamSynchronize(h->s.stream));
    if (t) *t = h->s.t;
    return QSLBM_OK;
}

int qslbm_set_state(qslbm_handle* h, const double* rho, const double* u, const double* b, int64_t t) {
    if (!h || t < 0) return bad_argument("qslbm_set_state: NULL handle or negative time");
    return set_fields(h->s, rho, u, b, t);
}

int qslbm_step_host(qslbm_handle* h, const double* rho_in, const double* u_in, const double* b_in, int64_t t_in,
                    int64_t nsteps, double* rho_out, double* u_out, double* b_out, qslbm_obs* obs) {
    if (!h) return bad_argument("qslbm_step_host: NULL handle");
    int rc = set_fields(h->s, rho_in, u_in, b_in, t_in);
    if (rc) return rc;
    if ((rc = step_impl(h->s, nsteps))) return rc;
    return qslbm_observables(h, obs, rho_out, u_out, b_out);
}

int qslbm_sync(qslbm_handle* h) {
    if (!h) return bad_argument("qslbm_sync: NULL handle");
    QCHK(cudaStreamSynchronize(h->s.stream));
    QCHK(cudaGetLastError());
    return check_resident(h->s);
}

int qslbm_destroy(qslbm_handle* h) {
    if (!h) return bad_argument("qslbm_destroy: NULL handle");
    cudaError_t e = cudaStreamSynchronize(h->s.stream);
    release(h->s);
    delete h;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return QSLBM_OK;
}

const char* qslbm_strerror(int code) {
    switch (code) {
        case QSLBM_OK: return "ok";
        case QSLBM_EINVAL: return "invalid argument";
        case QSLBM_ENOMEM: return "out of memory";
        case QSLBM_ECUDA: return "CUDA error";
        case QSLBM_EUNSTABLE: return "non-finite field value";
        case QSLBM_ETIMEOUT: return "timed out: step cap reached before the stop tolerance, or a bounded device wait gave up";
        case QSLBM_EBUDGET: return "request exceeds the device-memory budget";
        case QSLBM_ENOTFOUND: return "unknown request";
        case QSLBM_EARCH: return "device is not sm_103";
        default: return "unknown error";
    }
}

const char* qslbm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
