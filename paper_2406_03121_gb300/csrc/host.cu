// Host runtime of the library: basis construction, primitive-pair tables, Schwarz factors,
// quartet bins and the C ABI entry points of include/mess.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include <cuda_profiler_api.h>
#include <cstdlib>

#include "mess_internal.h"

// ------------------------------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void mess_set_error(const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

extern "C" const char* mess_last_error(void) { return g_last_error.c_str(); }

// ------------------------------------------------------------------------------------------ phase timing
static double wall_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

PhaseTimer::PhaseTimer(cudaStream_t stream) : s(stream)
{
    const char* e = getenv("MESS_TIMING");
    on = e && e[0] == '1';
    t = on ? wall_ms() : 0.0;
}

void PhaseTimer::mark(const char* label)
{
    if (!on) return;
    cudaStreamSynchronize(s);
    const double now = wall_ms();
    fprintf(stderr, "[mess] %s: %.2f ms\n", label, now - t);
    t = now;
}

// ------------------------------------------------------------------------------------------ basis file
namespace {

const char* kSymbols[] = {"", "H", "He", "Li", "Be", "B", "C", "N", "O", "F", "Ne"};

struct FileShell { int l; std::vector<double> a, d; };

bool parse_basis_file(const char* path, std::map<std::string, std::vector<FileShell>>& out)
{
    std::ifstream in(path);
    if (!in) { mess_set_error("cannot open basis file '%s'", path ? path : "(null)"); return false; }
    std::string line;
    std::vector<FileShell>* cur = nullptr;
    int lineno = 0;
    auto strip = [](std::string s) {
        size_t h = s.find('#');
        if (h != std::string::npos) s = s.substr(0, h);
        return s;
    };
    while (std::getline(in, line)) {
        ++lineno;
        line = strip(line);
        std::istringstream ss(line);
        std::string tok;
        if (!(ss >> tok)) continue;
        if (tok == "element") {
            std::string sym;
            if (!(ss >> sym)) { mess_set_error("%s:%d: element without symbol", path, lineno); return false; }
            cur = &out[sym];
            continue;
        }
        if (!cur) { mess_set_error("%s:%d: shell before any element line", path, lineno); return false; }
        int nprim = 0;
        if (!(ss >> nprim) || nprim <= 0 || nprim > 64) {
            mess_set_error("%s:%d: bad primitive count", path, lineno);
            return false;
        }
        std::string kind = tok;
        for (auto& c : kind) c = (char)toupper(c);
        bool sp = kind == "SP";
        int l = kind == "S" ? 0 : kind == "P" ? 1 : kind == "D" ? 2 : (sp ? 0 : -1);
        if (l < 0) { mess_set_error("%s:%d: unsupported shell type '%s'", path, lineno, tok.c_str()); return false; }
        FileShell s0{l, {}, {}}, s1{1, {}, {}};
        for (int k = 0; k < nprim; ++k) {
            std::string pl;
            do {
                if (!std::getline(in, pl)) { mess_set_error("%s: truncated shell", path); return false; }
                ++lineno;
                pl = strip(pl);
            } while (pl.find_first_not_of(" \t\r") == std::string::npos);
            std::istringstream ps(pl);
            double a, c0, c1 = 0.0;
            if (!(ps >> a >> c0) || (sp && !(ps >> c1)) || !(a > 0.0)) {
                mess_set_error("%s:%d: bad primitive line", path, lineno);
                return false;
            }
            s0.a.push_back(a); s0.d.push_back(c0);
            if (sp) { s1.a.push_back(a); s1.d.push_back(c1); }
        }
        cur->push_back(s0);
        if (sp) cur->push_back(s1);
    }
    return true;
}

double dfact(int k)
{
    double r = 1.0;
    while (k > 1) { r *= k; k -= 2; }
    return r;
}

int ncart(int l) { return (l + 1) * (l + 2) / 2; }

int pclass_of(int la, int lb)   // la >= lb
{
    static const int tab[3][3] = {{0, -1, -1}, {1, 2, -1}, {3, 4, 5}};
    return tab[la][lb];
}

// primitive-count group of a pair (lists are split so a launch's lanes run similar primitive loops)
int prim_group(int npp) { return npp <= 3 ? 0 : (npp <= 12 ? 1 : 2); }

int qclass_of(int p1, int p2)   // p1 >= p2
{
    return p1 * (p1 + 1) / 2 + p2;
}

// Contraction coefficients of one shell: each primitive normalised for its x^l component and the
// contraction renormalised so that the contracted x^l function has unit norm.
void normalise_shell(HostShell& s, const std::vector<double>& d)
{
    const int l = s.l;
    const double pi = M_PI;
    std::vector<double> c(s.K);
    for (int k = 0; k < s.K; ++k) {
        const double a = s.alpha[k];
        c[k] = d[k] * pow(2.0 * a / pi, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact(2 * l - 1));
    }
    double S = 0.0;
    for (int i = 0; i < s.K; ++i)
        for (int j = 0; j < s.K; ++j) {
            const double p = s.alpha[i] + s.alpha[j];
            S += c[i] * c[j] * pow(pi / p, 1.5) * dfact(2 * l - 1) / pow(2.0 * p, l);
        }
    s.coef.resize(s.K);
    for (int k = 0; k < s.K; ++k) s.coef[k] = c[k] / sqrt(S);
}

}  // namespace

// ------------------------------------------------------------------------------------------ bins
mess_status mess_ensure_bins(mess_basis* b, double tau, double tau64, int split)
{
    BinSet& B = b->bins;
    if (B.tau == tau && B.tau64 == tau64 && B.split == split && B.active_version == b->active_version) return MESS_OK;
    B.parts.clear();
    // per ket list (pair class x primitive group): Q, and prefix sums of unique function pairs and of
    // primitive pairs, in list order
    const int NL = MESS_NUM_PCLASS * MESS_NGROUP;
    std::vector<std::vector<long long>> fpre_l(NL), ppre_l(NL);
    for (int Lk = 0; Lk < NL; ++Lk) {
        const std::vector<int>& kl = b->class_list[Lk];
        const int nk = (int)kl.size();
        fpre_l[Lk].assign(nk + 1, 0);
        ppre_l[Lk].assign(nk + 1, 0);
        for (int j = 0; j < nk; ++j) {
            const int pk = kl[j];
            const int nc = ncart(b->shells[b->pair_a[pk]].l), nd = ncart(b->shells[b->pair_b[pk]].l);
            const long long nfp = b->pair_a[pk] == b->pair_b[pk] ? (long long)nc * (nc + 1) / 2 : (long long)nc * nd;
            fpre_l[Lk][j + 1] = fpre_l[Lk][j] + nfp;
            ppre_l[Lk][j + 1] = ppre_l[Lk][j] + b->pp_n[pk];
        }
    }
    // One task per unordered pair of lists (list g1 x list g2 for g1 > g2, the triangle for g1 == g2
    // within one pair class); each builds its parts (FP64-class / reduced-precision split) into its
    // own arrays.  Tasks are independent and run on host threads; the parts are concatenated in task
    // order, so the bins do not depend on the threading.
    struct Task { int p1, p2, g1, g2; std::vector<BinPart> parts; std::vector<int> bra, kbeg; std::vector<long long> offs; };
    std::vector<Task> tasks;
    for (int p1 = 0; p1 < MESS_NUM_PCLASS; ++p1)
        for (int p2 = 0; p2 <= p1; ++p2)
            for (int g1 = 0; g1 < MESS_NGROUP; ++g1)
                for (int g2 = 0; g2 < MESS_NGROUP; ++g2) {
                    if (p1 == p2 && g2 > g1) continue;
                    if (b->class_list[p1 * MESS_NGROUP + g1].empty() || b->class_list[p2 * MESS_NGROUP + g2].empty()) continue;
                    tasks.push_back(Task{p1, p2, g1, g2, {}, {}, {}, {}});
                }
    auto run_task = [&](Task& T) {
        const int p1 = T.p1, p2 = T.p2, g1 = T.g1, g2 = T.g2;
        const int L1 = p1 * MESS_NGROUP + g1, L2 = p2 * MESS_NGROUP + g2;
        const std::vector<int>& bl = b->class_list[L1];
        const std::vector<long long>& fpre = fpre_l[L2];
        const std::vector<long long>& ppre = ppre_l[L2];
        const std::vector<int>& kl = b->class_list[L2];
        const bool same = p1 == p2 && g1 == g2;
        std::vector<int>& bra = T.bra;
        std::vector<int>& kbeg = T.kbeg;
        std::vector<long long>& offs = T.offs;
        const int nparts = split == 2 ? 2 : 1;
        for (int part = 0; part < nparts; ++part) {
            const int fp64 = split == 0 ? 1 : (split == 1 ? 0 : (part == 0 ? 1 : 0));
            BinPart bp;
            bp.qclass = qclass_of(p1, p2);
            bp.fp64 = fp64;
            bp.bra_off = (int)bra.size();
            bp.ket_list = L2;
            bp.offs_off = offs.size();
            bp.total = 0;
            bp.fn_quartets = 0;
            bp.prim_quartets = 0;
            for (int m = 0; m < b->nmol; ++m) {
                if (!b->active[m]) continue;
                const int bs0 = b->class_seg[L1][m], bs1 = b->class_seg[L1][m + 1];
                const int ks0 = b->class_seg[L2][m], ks1 = b->class_seg[L2][m + 1];
                if (bs1 == bs0 || ks1 == ks0) continue;
                // kets j in [ks0, ks1) (Q descending) with qi * Q_j >= t: a prefix of the segment
                auto count_ge = [&](double qi, double t) -> int {
                    if (t <= 0.0) return ks1 - ks0;
                    int lo = ks0, hi = ks1;
                    while (lo < hi) {
                        const int mid = (lo + hi) / 2;
                        if (qi * b->Q[kl[mid]] >= t) lo = mid + 1; else hi = mid;
                    }
                    return lo - ks0;
                };
                for (int i = bs0; i < bs1; ++i) {
                    const int il = i - bs0;
                    const int pb = bl[i];
                    const double qi = b->Q[pb];
                    int cnt = count_ge(qi, tau);
                    if (same) cnt = std::min(cnt, il + 1);
                    int beg = 0, end = cnt;
                    if (split == 2) {
                        const int c64 = tau64 > 0.0 ? std::min(count_ge(qi, tau64), cnt) : 0;
                        if (part == 0) end = c64; else beg = c64;
                    }
                    if (end <= beg) continue;
                    bra.push_back(pb);
                    kbeg.push_back(ks0 + beg);
                    offs.push_back(bp.total);
                    bp.total += end - beg;
                    const int na = ncart(b->shells[b->pair_a[pb]].l), nb = ncart(b->shells[b->pair_b[pb]].l);
                    const long long nfb = b->pair_a[pb] == b->pair_b[pb] ? (long long)na * (na + 1) / 2 : (long long)na * nb;
                    bp.fn_quartets += nfb * (fpre[ks0 + end] - fpre[ks0 + beg]);
                    if (same && beg <= il && il < end) bp.fn_quartets += nfb * (nfb + 1) / 2 - nfb * nfb;
                    bp.prim_quartets += (long long)b->pp_n[pb] * (ppre[ks0 + end] - ppre[ks0 + beg]);
                }
            }
            bp.nbra = (int)bra.size() - bp.bra_off;
            offs.push_back(bp.total);
            // heavily contracted quartets: split the primitive loop over 8 lanes
            const bool straight = MESS_QCLASS[bp.qclass].straight != 0;
            const double avg = bp.total > 0 ? (double)bp.prim_quartets / (double)bp.total : 0.0;
            // lanes per quartet (the choice when the kernels are not autotuned).  FP64-class parts: 8 for
            // long primitive loops, 4 for medium loops of parts too small to fill the GPU one thread per
            // quartet.  Reduced-precision parts: one thread per quartet unless the part is small and its
            // loops long - with G lanes only one lane in G digests, and for the small classes the
            // digestion is most of the per-quartet work (measured on STO-3G alkanes, 81 primitive
            // quartets per shell quartet: one thread per quartet 2.2x faster than 8 lanes).
            if (!straight) bp.G = 1;
            else if (fp64) bp.G = avg >= 24.0 ? 8 : ((avg >= 6.0 && bp.total < (1LL << 18)) ? 4 : 1);
            else bp.G = (avg >= 6.0 && bp.total < (1LL << 15)) ? 4 : 1;
            // warp per quartet: always for the op-program classes; for small FP64 parts of the classes
            // with at least 40 VRR entries (too few quartets to fill the GPU one thread each:
            // measured better below about 2e6 quartets x VRR entries, worse above)
            const double work = (double)bp.total * MESS_QCLASS[bp.qclass].nvrr;
            bp.team = (!straight || (fp64 && MESS_QCLASS[bp.qclass].team && bp.G == 1 && work < 2e6)) ? 1 : 0;
            if (bp.nbra > 0) T.parts.push_back(bp);
            else offs.resize(bp.offs_off);
        }
    };
    {
        std::atomic<size_t> next(0);
        auto worker = [&]() {
            for (size_t t; (t = next.fetch_add(1)) < tasks.size();) run_task(tasks[t]);
        };
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int nthr = std::max(1, std::min({hw, 32, (int)tasks.size()}));
        std::vector<std::thread> workers;
        for (int t = 1; t < nthr; ++t) workers.emplace_back(worker);
        worker();
        for (auto& w : workers) w.join();
    }
    std::vector<int> bra, kbeg;
    std::vector<long long> offs;
    for (Task& T : tasks) {
        for (BinPart bp : T.parts) {
            bp.bra_off += (int)bra.size();
            bp.offs_off += offs.size();
            B.parts.push_back(bp);
        }
        bra.insert(bra.end(), T.bra.begin(), T.bra.end());
        kbeg.insert(kbeg.end(), T.kbeg.begin(), T.kbeg.end());
        offs.insert(offs.end(), T.offs.begin(), T.offs.end());
    }
    tasks.clear();
    // per part, the bra of every 32nd quartet
    std::vector<int> seg;
    for (BinPart& p : B.parts) {
        p.seg_off = seg.size();
        const long long* po = offs.data() + p.offs_off;   // [nbra + 1]
        int i = 0;
        for (long long q = 0; q < p.total; q += 32) {
            while (i + 1 < p.nbra && po[i + 1] <= q) ++i;
            seg.push_back(i);
        }
    }
    if (B.bra.upload(bra) != cudaSuccess || B.kbeg.upload(kbeg) != cudaSuccess || B.offs.upload(offs) != cudaSuccess ||
        B.seg.upload(seg) != cudaSuccess) {
        mess_set_error("uploading quartet bins failed");
        B.tau = -1.0;
        return MESS_ECUDA;
    }
    // the reduced-precision density copies (and their reuse event) come with the bins, so that a
    // build with ready bins allocates nothing
    if (split != 0) {
        cudaError_t e = cudaSuccess;
        if (b->d_D32.n != (size_t)b->packed) e = b->d_D32.alloc((size_t)b->packed);
        if (e == cudaSuccess && split == 2 && b->d_Ddf.n != (size_t)b->packed) e = b->d_Ddf.alloc((size_t)b->packed);
        if (e == cudaSuccess && !b->dconv_free) e = cudaEventCreateWithFlags(&b->dconv_free, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            mess_set_error("density copies: %s", cudaGetErrorString(e));
            B.tau = -1.0;
            return MESS_ECUDA;
        }
    }
    B.tau = tau;
    B.tau64 = tau64;
    B.split = split;
    B.active_version = b->active_version;
    B.generation += 1;
    mess_free_jk_graphs(b);
    return MESS_OK;
}

// ------------------------------------------------------------------------------------------ streams
// Per-device pool of non-blocking streams: the class launches of one J/K build fork from the
// caller's stream, run concurrently (most of them are small), and join back before the
// symmetrisation.  Fork/join is by events, so a captured caller stream captures the whole build.
// The number of streams is MESS_JK_STREAMS from the environment when the pool is created (8..64),
// else 16.
#define MESS_MAX_STREAMS 64
#define MESS_DEFAULT_STREAMS 16
#define MESS_TUNE_COPIES 8   // concurrent copies of a candidate kernel timed by the autotuner
struct StreamPool {
    bool init = false;
    int n = MESS_DEFAULT_STREAMS;
    cudaStream_t s[MESS_MAX_STREAMS];
    cudaEvent_t fork, join[MESS_MAX_STREAMS];
    cudaStream_t capture;   // private stream on which J/K graphs are captured
    std::mutex mu;
};
static StreamPool g_pools[64];

static cudaError_t get_pool(StreamPool** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    StreamPool& P = g_pools[dev];
    std::lock_guard<std::mutex> lk(P.mu);
    if (!P.init) {
        const char* env = getenv("MESS_JK_STREAMS");
        int n = env ? atoi(env) : MESS_DEFAULT_STREAMS;
        P.n = std::max(MESS_TUNE_COPIES, std::min(MESS_MAX_STREAMS, n));
        for (int i = 0; i < P.n; ++i) {
            if ((e = cudaStreamCreateWithFlags(&P.s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaStreamCreateWithFlags(&P.capture, cudaStreamNonBlocking)) != cudaSuccess) return e;
        P.init = true;
    }
    *out = &P;
    return cudaSuccess;
}

static BinLaunch bin_launch(const mess_basis* b, const BinPart& p)
{
    BinLaunch L;
    L.bra = b->bins.bra.p + p.bra_off;
    L.kbeg = b->bins.kbeg.p + p.bra_off;
    L.offs = b->bins.offs.p + p.offs_off;
    L.seg = b->bins.seg.p + p.seg_off;
    L.ket = b->d_class_list[p.ket_list].p;
    L.ketrec = b->d_ketrec[p.ket_list].p;
    L.nbra = p.nbra;
    L.total = p.total;
    return L;
}

// ------------------------------------------------------------------------------------------ create
// Append one molecule (atoms and already normalised shells) to a basis under construction.
static void add_molecule(mess_basis* b, const std::vector<int>& Z, const std::vector<double>& xyz,
                         const std::vector<HostShell>& shells)
{
    const int m = (int)b->mol_nbf.size();
    const int atom0 = b->natom;
    b->mol_atom_off.push_back(atom0);
    b->mol_atom_n.push_back((int)Z.size());
    b->mol_shell_off.push_back((int)b->shells.size());
    b->mol_shell_n.push_back((int)shells.size());
    int fl = 0, nel = 0;
    for (HostShell s : shells) {
        s.atom = s.atom + atom0;
        s.mol = m;
        s.fl = fl;
        s.f0 = b->nbf + fl;
        fl += ncart(s.l);
        b->shells.push_back(s);
    }
    for (int z : Z) nel += z;
    b->Z.insert(b->Z.end(), Z.begin(), Z.end());
    b->xyz.insert(b->xyz.end(), xyz.begin(), xyz.end());
    b->natom += (int)Z.size();
    b->mol_base.push_back(b->packed);
    b->packed += (long long)fl * fl;
    b->mol_nbf.push_back(fl);
    b->mol_nelec.push_back(nel);
    b->nbf += fl;
    b->nelec += nel;
    b->max_nbf = std::max(b->max_nbf, fl);
    b->nmol = m + 1;
    b->active.push_back(1);
}

// Shells of one structure from a parsed basis file, normalised (molecule-local atom indices).
static mess_status shells_from_file(int natom, const int* Z, const double* xyz,
                                    const std::map<std::string, std::vector<FileShell>>& data,
                                    const char* basis_file, std::vector<HostShell>& out)
{
    for (int a = 0; a < natom; ++a) {
        const int z = Z[a];
        if (z <= 0 || z > 10) { mess_set_error("unsupported atomic number %d", z); return MESS_EINVAL; }
        auto it = data.find(kSymbols[z]);
        if (it == data.end()) { mess_set_error("element %s not in basis file %s", kSymbols[z], basis_file); return MESS_EINVAL; }
        for (const FileShell& fs : it->second) {
            if (fs.l > MESS_LMAX) { mess_set_error("angular momentum %d not supported", fs.l); return MESS_EINVAL; }
            HostShell s;
            s.l = fs.l;
            s.K = (int)fs.a.size();
            s.atom = a;
            s.f0 = s.fl = 0;
            s.mol = 0;
            for (int x = 0; x < 3; ++x) s.R[x] = xyz[3 * a + x];
            s.alpha = fs.a;
            normalise_shell(s, fs.d);
            out.push_back(s);
        }
    }
    return MESS_OK;
}

static mess_status build_pairs(mess_basis* b)
{
    // per-function component scale sqrt((2L-1)!! / ((2l-1)!!(2m-1)!!(2n-1)!!)) and local index
    b->fscale.clear();
    b->f_local.clear();
    for (const HostShell& s : b->shells) {
        int k = 0;
        for (int lx = s.l; lx >= 0; --lx)
            for (int ly = s.l - lx; ly >= 0; --ly, ++k) {
                const int lz = s.l - lx - ly;
                b->fscale.push_back(sqrt(dfact(2 * s.l - 1) / (dfact(2 * lx - 1) * dfact(2 * ly - 1) * dfact(2 * lz - 1))));
                b->f_local.push_back(s.fl + k);
            }
    }
    const double kpref = sqrt(2.0) * pow(M_PI, 1.25);
    // Primitive-pair screening.  The product of two primitives a, b (coefficients c_a, c_b) is a
    // Gaussian distribution of total weight S_ab = |c_a c_b| exp(-alpha beta/zeta |AB|^2) (pi/zeta)^(3/2);
    // the Coulomb integral of two such s-type distributions is S_ab S_cd 2 sqrt(rho/pi) F_0 <=
    // M_ab M_cd with M = sqrt(2) (zeta/pi)^(1/4) S.  A primitive pair whose M times the largest M of
    // the basis is below MESS_PRIM_EPS contributes nothing measurable to any integral (the margin
    // of MESS_PRIM_EPS covers the polynomial factors of p and d functions and the number of
    // primitive quartets of a shell quartet), and is left out of the pair's primitive list.
    auto prim_weight = [](const HostShell& sa, const HostShell& sb, int i, int j, double ab2) {
        const double al = sa.alpha[i], be = sb.alpha[j], z = al + be;
        const double u = M_PI / z;   // M = sqrt(2) (zeta/pi)^(1/4) (pi/zeta)^(3/2) |c_a c_b| exp(..) = sqrt(2) u^(5/4) ...
        return sqrt(2.0) * u * sqrt(sqrt(u)) * fabs(sa.coef[i] * sb.coef[j]) * exp(-al * be / z * ab2);
    };
    double Mmax = 0.0;
    for (int m = 0; m < b->nmol; ++m) {
        const int s0 = b->mol_shell_off[m], s1 = s0 + b->mol_shell_n[m];
        for (int A = s0; A < s1; ++A)       // the scale: the largest weight of a primitive with itself
            for (int i = 0; i < b->shells[A].K; ++i)
                for (int j = 0; j < b->shells[A].K; ++j)
                    Mmax = std::max(Mmax, prim_weight(b->shells[A], b->shells[A], i, j, 0.0));
    }
    // The pairs of molecules [m0, m1): shell pairs A >= B (canonical order) of each molecule, with
    // their kept primitive pairs.  Molecules are independent, so contiguous molecule ranges are built
    // on host threads and concatenated in molecule order (the result does not depend on the split).
    struct Chunk {
        std::vector<int> pa, pb, pcls, pmol, pn, fa, fb, same;
        std::vector<double> AB, Ccen;
        std::vector<float> ABf, Cf;
        std::vector<PrimPairRec<double>> pp64;
        std::vector<PrimPairRec<float>> pp32;
        std::vector<PrimPairRec<df32>> ppdf;
    };
    auto build_chunk = [&](int m0, int m1, Chunk& c) {
        std::vector<double> wts;
        for (int m = m0; m < m1; ++m) {
            const int s0 = b->mol_shell_off[m], s1 = s0 + b->mol_shell_n[m];
            for (int A = s0; A < s1; ++A) {
                for (int B = s0; B < s1; ++B) {
                    const HostShell& sa = b->shells[A];
                    const HostShell& sb = b->shells[B];
                    const bool canonical = sa.l > sb.l || (sa.l == sb.l && A >= B);
                    if (!canonical) continue;
                    c.pa.push_back(A);
                    c.pb.push_back(B);
                    c.pcls.push_back(pclass_of(sa.l, sb.l));
                    c.pmol.push_back(m);
                    double ab2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        const double abx = sa.R[x] - sb.R[x];
                        ab2 += abx * abx;
                        c.AB.push_back(abx);
                        c.ABf.push_back((float)abx);
                        c.Ccen.push_back(sa.R[x]);
                    }
                    for (int x = 0; x < 3; ++x) c.Cf.push_back((float)sa.R[x]);
                    for (int x = 0; x < 3; ++x) c.Cf.push_back((float)(sa.R[x] - (double)(float)sa.R[x]));
                    // kept primitive pairs; at least the heaviest one, so that no pair is empty
                    int npp = 0, heavy = 0;
                    double wmax = -1.0;
                    wts.resize((size_t)sa.K * sb.K);
                    for (int i = 0; i < sa.K; ++i)
                        for (int j = 0; j < sb.K; ++j) {
                            const double w = prim_weight(sa, sb, i, j, ab2);
                            wts[(size_t)i * sb.K + j] = w;
                            if (w > wmax) { wmax = w; heavy = i * sb.K + j; }
                        }
                    for (int i = 0; i < sa.K; ++i)
                        for (int j = 0; j < sb.K; ++j) {
                            if (wts[(size_t)i * sb.K + j] * Mmax < MESS_PRIM_EPS && i * sb.K + j != heavy) continue;
                            ++npp;
                            const double al = sa.alpha[i], be = sb.alpha[j], z = al + be;
                            PrimPairRec<double> r{};
                            r.v[0] = z;
                            for (int x = 0; x < 3; ++x) {
                                const double P = (al * sa.R[x] + be * sb.R[x]) / z;
                                r.v[1 + x] = P - sa.R[x];
                            }
                            r.v[4] = kpref * sa.coef[i] * sb.coef[j] * exp(-al * be / z * ab2) / z;
                            r.v[5] = 0.5 / z;
                            c.pp64.push_back(r);
                            PrimPairRec<float> f{};
                            PrimPairRec<df32> g;
                            for (int k = 0; k < 8; ++k) {
                                f.v[k] = (float)r.v[k];
                                g.v[k].hi = (float)r.v[k];
                                g.v[k].lo = (float)(r.v[k] - (double)g.v[k].hi);
                            }
                            c.pp32.push_back(f);
                            c.ppdf.push_back(g);
                        }
                    c.pn.push_back(npp);
                    c.fa.push_back(sa.fl);
                    c.fb.push_back(sb.fl);
                    c.same.push_back(A == B ? 1 : 0);
                }
            }
        }
    };
    // molecule ranges of about equal work (shells squared) for the host threads
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nthr = std::max(1, std::min({hw, 32, b->nmol}));
    std::vector<int> cut(1, 0);
    {
        double tot = 0.0, acc = 0.0;
        for (int m = 0; m < b->nmol; ++m) tot += (double)b->mol_shell_n[m] * b->mol_shell_n[m];
        for (int m = 0; m < b->nmol && (int)cut.size() < nthr; ++m) {
            acc += (double)b->mol_shell_n[m] * b->mol_shell_n[m];
            if (acc >= tot * (double)cut.size() / nthr && m + 1 < b->nmol) cut.push_back(m + 1);
        }
        cut.push_back(b->nmol);
    }
    std::vector<Chunk> chunks(cut.size() - 1);
    {
        std::vector<std::thread> workers;
        for (size_t t = 1; t < chunks.size(); ++t)
            workers.emplace_back(build_chunk, cut[t], cut[t + 1], std::ref(chunks[t]));
        build_chunk(cut[0], cut[1], chunks[0]);
        for (auto& w : workers) w.join();
    }
    // concatenation in molecule order; the primitive records go to the device chunk by chunk
    std::vector<double> AB, Ccen;
    std::vector<float> ABf, Cf;
    std::vector<int> fa, fb, same;
    size_t npp_tot = 0;
    for (const Chunk& c : chunks) {
        for (size_t k = 0; k < c.pa.size(); ++k) {
            b->pp_off.push_back((int)npp_tot);
            npp_tot += (size_t)c.pn[k];
        }
        b->pair_a.insert(b->pair_a.end(), c.pa.begin(), c.pa.end());
        b->pair_b.insert(b->pair_b.end(), c.pb.begin(), c.pb.end());
        b->pair_class.insert(b->pair_class.end(), c.pcls.begin(), c.pcls.end());
        b->pair_mol.insert(b->pair_mol.end(), c.pmol.begin(), c.pmol.end());
        b->pp_n.insert(b->pp_n.end(), c.pn.begin(), c.pn.end());
        AB.insert(AB.end(), c.AB.begin(), c.AB.end());
        Ccen.insert(Ccen.end(), c.Ccen.begin(), c.Ccen.end());
        ABf.insert(ABf.end(), c.ABf.begin(), c.ABf.end());
        Cf.insert(Cf.end(), c.Cf.begin(), c.Cf.end());
        fa.insert(fa.end(), c.fa.begin(), c.fa.end());
        fb.insert(fb.end(), c.fb.begin(), c.fb.end());
        same.insert(same.end(), c.same.begin(), c.same.end());
    }
    if (npp_tot > (size_t)INT32_MAX) { mess_set_error("too many primitive pairs (%zu)", npp_tot); return MESS_EINVAL; }
    b->npair = (int)b->pair_a.size();
    MESS_CUDA_TRY(b->d_pp64.alloc(npp_tot));
    MESS_CUDA_TRY(b->d_pp32.alloc(npp_tot));
    MESS_CUDA_TRY(b->d_ppdf.alloc(npp_tot));
    {
        size_t off = 0;
        for (const Chunk& c : chunks) {
            const size_t k = c.pp64.size();
            if (k) {
                MESS_CUDA_TRY(cudaMemcpy(b->d_pp64.p + off, c.pp64.data(), k * sizeof(c.pp64[0]), cudaMemcpyHostToDevice));
                MESS_CUDA_TRY(cudaMemcpy(b->d_pp32.p + off, c.pp32.data(), k * sizeof(c.pp32[0]), cudaMemcpyHostToDevice));
                MESS_CUDA_TRY(cudaMemcpy(b->d_ppdf.p + off, c.ppdf.data(), k * sizeof(c.ppdf[0]), cudaMemcpyHostToDevice));
            }
            off += k;
        }
    }
    chunks.clear();
    MESS_CUDA_TRY(b->d_pp_off.upload(b->pp_off));
    MESS_CUDA_TRY(b->d_pp_n.upload(b->pp_n));
    MESS_CUDA_TRY(b->d_AB.upload(AB));
    MESS_CUDA_TRY(b->d_Ccen.upload(Ccen));
    MESS_CUDA_TRY(b->d_ABf.upload(ABf));
    MESS_CUDA_TRY(b->d_Cf.upload(Cf));
    MESS_CUDA_TRY(b->d_fa.upload(fa));
    MESS_CUDA_TRY(b->d_fb.upload(fb));
    MESS_CUDA_TRY(b->d_same.upload(same));
    // the per-pair records the J/K kernels read for the ket of a quartet
    b->pair_rec.assign(b->npair, KetRec{});
    for (int p = 0; p < b->npair; ++p) {
        KetRec& r = b->pair_rec[p];
        r.pp_off = b->pp_off[p];
        r.pp_n = b->pp_n[p];
        r.fab = fa[p] | (fb[p] << 16);
        r.flags = same[p] | (b->pair_mol[p] << 1);
        for (int x = 0; x < 3; ++x) {
            r.C[x] = Ccen[3 * p + x];
            r.AB[x] = AB[3 * p + x];
            r.Cf[x] = Cf[6 * p + x];
            r.Cf[3 + x] = Cf[6 * p + 3 + x];
            r.ABf[x] = ABf[3 * p + x];
        }
        r.pair = p;
    }
    MESS_CUDA_TRY(b->d_pair_rec.upload(b->pair_rec));
    std::vector<double> tab;
    mess_boys_table(tab, MESS_BOYS_NROW, MESS_BOYS_DT);
    MESS_CUDA_TRY(b->d_boys64.upload(tab));
    std::vector<float> tab32(tab.begin(), tab.end());
    MESS_CUDA_TRY(b->d_boys32.upload(tab32));
    // FP32 rows per order L on the finer grid, one float4 per row: F_L, F_L+1, F_L+2, exp(-T_k)
    std::vector<double> fine;
    mess_boys_table(fine, MESS_BOYS32_NROW, MESS_BOYS32_DT);
    std::vector<float4> tabv((size_t)MESS_BOYS_NL * MESS_BOYS32_NROW);
    for (int L = 0; L < MESS_BOYS_NL; ++L)
        for (int k = 0; k < MESS_BOYS32_NROW; ++k) {
            const double* row = fine.data() + (size_t)k * MESS_BOYS_NCOL;
            tabv[(size_t)L * MESS_BOYS32_NROW + k] =
                make_float4((float)row[L], (float)row[L + 1], (float)row[L + 2], (float)row[MESS_BOYS_NF]);
        }
    MESS_CUDA_TRY(b->d_boys32v.upload(tabv));
    std::vector<float2> tabdf(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) {
        tabdf[i].x = (float)tab[i];
        tabdf[i].y = (float)(tab[i] - (double)tabdf[i].x);
    }
    MESS_CUDA_TRY(b->d_boysdf.upload(tabdf));
    MESS_CUDA_TRY(b->d_pair_mol.upload(b->pair_mol));
    MESS_CUDA_TRY(b->d_mol_base.upload(b->mol_base));
    MESS_CUDA_TRY(b->d_mol_n.upload(b->mol_nbf));
    MESS_CUDA_TRY(b->d_mol_atom_off.upload(b->mol_atom_off));
    MESS_CUDA_TRY(b->d_mol_atom_n.upload(b->mol_atom_n));
    MESS_CUDA_TRY(b->d_f_local.upload(b->f_local));
    b->P64.pp = b->d_pp64.p;
    b->P32.pp = b->d_pp32.p;
    b->P64.pp_off = b->P32.pp_off = b->d_pp_off.p;
    b->P64.pp_n = b->P32.pp_n = b->d_pp_n.p;
    b->P64.AB = b->P32.AB = b->d_AB.p;
    b->P64.fa = b->P32.fa = b->d_fa.p;
    b->P64.fb = b->P32.fb = b->d_fb.p;
    b->P64.same = b->P32.same = b->d_same.p;
    b->P64.C = b->P32.C = b->d_Ccen.p;
    b->P64.Cf = b->P32.Cf = b->d_Cf.p;
    b->P64.ABf = b->P32.ABf = b->d_ABf.p;
    b->P64.mol = b->P32.mol = b->d_pair_mol.p;
    b->P64.rec = b->P32.rec = b->Pdf.rec = b->d_pair_rec.p;
    b->P64.mbase = b->P32.mbase = b->d_mol_base.p;
    b->P64.mn = b->P32.mn = b->d_mol_n.p;
    b->P64.boys64 = b->P32.boys64 = b->d_boys64.p;
    b->P64.boys32 = b->P32.boys32 = b->d_boys32.p;
    b->P64.boys32v = b->P32.boys32v = b->d_boys32v.p;
    b->P64.boysdf = b->P32.boysdf = b->d_boysdf.p;
    // the double-float table shares every per-pair array with the others
    b->Pdf.pp = b->d_ppdf.p;
    b->Pdf.pp_off = b->P64.pp_off; b->Pdf.pp_n = b->P64.pp_n; b->Pdf.AB = b->P64.AB; b->Pdf.fa = b->P64.fa;
    b->Pdf.fb = b->P64.fb; b->Pdf.same = b->P64.same; b->Pdf.C = b->P64.C; b->Pdf.Cf = b->P64.Cf;
    b->Pdf.ABf = b->P64.ABf; b->Pdf.mol = b->P64.mol; b->Pdf.mbase = b->P64.mbase; b->Pdf.mn = b->P64.mn;
    b->Pdf.boys64 = b->d_boys64.p; b->Pdf.boys32 = b->d_boys32.p; b->Pdf.boysdf = b->d_boysdf.p;
    b->Pdf.boys32v = b->d_boys32v.p;
    // shells for the one-electron kernels
    std::vector<int> sl, sK, sf0, spoff;
    std::vector<double> sR, sal, sco;
    for (const HostShell& s : b->shells) {
        sl.push_back(s.l); sK.push_back(s.K); sf0.push_back(s.f0); spoff.push_back((int)sal.size());
        for (int x = 0; x < 3; ++x) sR.push_back(s.R[x]);
        sal.insert(sal.end(), s.alpha.begin(), s.alpha.end());
        sco.insert(sco.end(), s.coef.begin(), s.coef.end());
    }
    MESS_CUDA_TRY(b->d_shell_l.upload(sl));
    MESS_CUDA_TRY(b->d_shell_K.upload(sK));
    MESS_CUDA_TRY(b->d_shell_f0.upload(sf0));
    MESS_CUDA_TRY(b->d_shell_poff.upload(spoff));
    MESS_CUDA_TRY(b->d_shell_R.upload(sR));
    MESS_CUDA_TRY(b->d_shell_alpha.upload(sal));
    MESS_CUDA_TRY(b->d_shell_coef.upload(sco));
    MESS_CUDA_TRY(b->d_fscale.upload(b->fscale));
    MESS_CUDA_TRY(b->d_pair_a.upload(b->pair_a));
    MESS_CUDA_TRY(b->d_pair_b.upload(b->pair_b));
    MESS_CUDA_TRY(b->d_Z.upload(b->Z));
    MESS_CUDA_TRY(b->d_xyz.upload(b->xyz));
    return MESS_OK;
}

static mess_status build_schwarz(mess_basis* b)
{
    std::vector<int> lists[MESS_NUM_PCLASS];
    for (int p = 0; p < b->npair; ++p) lists[b->pair_class[p]].push_back(p);
    MESS_CUDA_TRY(b->d_Q.alloc((size_t)std::max(1, b->npair)));
    DevBuf<int> tmp[MESS_NUM_PCLASS];
    for (int c = 0; c < MESS_NUM_PCLASS; ++c) {
        if (lists[c].empty()) continue;
        MESS_CUDA_TRY(tmp[c].upload(lists[c]));
        ClassLaunchArgs a{};
        a.kind = MESS_KIND_SCHWARZ;
        a.pairs = tmp[c].p;
        a.npairs = (int)lists[c].size();
        a.P64_ptr = &b->P64;
        a.P32_ptr = &b->P32;
        a.out = b->d_Q.p;
        a.stream = 0;
        MESS_CUDA_TRY(MESS_CLASS_LAUNCHERS[qclass_of(c, c)](a));
    }
    MESS_CUDA_TRY(cudaDeviceSynchronize());
    b->Q.resize(b->npair);
    MESS_CUDA_TRY(cudaMemcpy(b->Q.data(), b->d_Q.p, sizeof(double) * b->npair, cudaMemcpyDeviceToHost));
    for (int p = 0; p < b->npair; ++p)
        if (!std::isfinite(b->Q[p])) { mess_set_error("non-finite Schwarz factor for pair %d", p); return MESS_ENUMERIC; }
    {
        // FP32 copy for the density-screening test (rounded up, so that the bound stays a bound)
        std::vector<float> qf(std::max(1, b->npair), 0.f);
        for (int p = 0; p < b->npair; ++p) qf[p] = nextafterf((float)b->Q[p], INFINITY);
        MESS_CUDA_TRY(b->d_Qf.upload(qf));
        b->P64.Qf = b->P32.Qf = b->Pdf.Qf = b->d_Qf.p;
    }
    // lists per (class, primitive-count group): per molecule, pairs sorted by Q descending
    for (int c = 0; c < MESS_NUM_PCLASS; ++c) {
        for (int g = 0; g < MESS_NGROUP; ++g) {
            std::vector<std::vector<int>> per(b->nmol);
            for (int p : lists[c])
                if (prim_group(b->pp_n[p]) == g) per[b->pair_mol[p]].push_back(p);
            std::vector<int> l;
            std::vector<int> seg(1, 0);
            for (int m = 0; m < b->nmol; ++m) {
                std::stable_sort(per[m].begin(), per[m].end(), [&](int x, int y) { return b->Q[x] > b->Q[y]; });
                l.insert(l.end(), per[m].begin(), per[m].end());
                seg.push_back((int)l.size());
            }
            const int L = c * MESS_NGROUP + g;
            b->class_list[L] = l;
            b->class_seg[L] = seg;
            MESS_CUDA_TRY(b->d_class_list[L].upload(l));
            std::vector<KetRec> rl(l.size());
            for (size_t k = 0; k < l.size(); ++k) rl[k] = b->pair_rec[l[k]];
            MESS_CUDA_TRY(b->d_ketrec[L].upload(rl));
        }
    }
    return MESS_OK;
}

void mess_free_basis(mess_basis* b)
{
    b->d_pp64.free(); b->d_pp32.free(); b->d_ppdf.free(); b->d_boysdf.free(); b->d_pp_off.free(); b->d_pp_n.free(); b->d_fa.free();
    b->d_fb.free(); b->d_same.free(); b->d_AB.free(); b->d_Ccen.free(); b->d_ABf.free(); b->d_Cf.free(); b->d_Q.free(); b->d_Qf.free(); b->d_boys64.free();
    b->d_boys32.free(); b->d_boys32v.free(); b->d_Z.free(); b->d_xyz.free(); b->d_shell_l.free(); b->d_shell_K.free();
    b->d_shell_f0.free(); b->d_shell_poff.free(); b->d_shell_R.free(); b->d_shell_alpha.free();
    b->d_shell_coef.free(); b->d_fscale.free(); b->d_pair_a.free(); b->d_pair_b.free();
    b->d_pair_mol.free(); b->d_mol_n.free(); b->d_mol_atom_off.free(); b->d_mol_atom_n.free();
    b->d_f_local.free(); b->d_mol_base.free();
    for (auto& d : b->d_class_list) d.free();
    for (auto& d : b->d_ketrec) d.free();
    b->d_pair_rec.free();
    b->bins.bra.free(); b->bins.kbeg.free(); b->bins.offs.free(); b->bins.seg.free();
    mess_free_jk_graphs(b);
    b->d_D32.free(); b->d_Ddf.free(); b->d_stage.free();
    mess_free_xc(b);
    if (b->dconv_free) cudaEventDestroy(b->dconv_free);
    b->dconv_free = nullptr;
}

extern "C" mess_status mess_basis_create(int natom, const int* Z, const double* xyz_bohr, const char* basis_file,
                                         mess_basis** out)
{
    if (!out) { mess_set_error("out is NULL"); return MESS_EINVAL; }
    *out = nullptr;
    if (natom <= 0 || !Z || !xyz_bohr || !basis_file) { mess_set_error("bad structure arguments"); return MESS_EINVAL; }
    for (int i = 0; i < 3 * natom; ++i)
        if (!std::isfinite(xyz_bohr[i])) { mess_set_error("non-finite coordinate"); return MESS_EINVAL; }
    std::map<std::string, std::vector<FileShell>> data;
    if (!parse_basis_file(basis_file, data)) return MESS_EINVAL;
    std::vector<HostShell> shells;
    mess_status st = shells_from_file(natom, Z, xyz_bohr, data, basis_file, shells);
    if (st != MESS_OK) return st;
    mess_basis* b = new (std::nothrow) mess_basis();
    if (!b) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    add_molecule(b, std::vector<int>(Z, Z + natom), std::vector<double>(xyz_bohr, xyz_bohr + 3 * natom), shells);
    *out = b;
    return MESS_OK;
}

mess_status mess_basis_gpu(mess_basis* b)
{
    if (!b) { mess_set_error("basis is NULL"); return MESS_EINVAL; }
    if (b->gpu_ready) return MESS_OK;
    mess_status st = build_pairs(b);
    if (st == MESS_OK) st = build_schwarz(b);
    if (st != MESS_OK) {
        // leave the basis as created (host data only) so that a later call can try again
        mess_free_basis(b);
        b->npair = 0;
        b->pair_a.clear(); b->pair_b.clear(); b->pair_class.clear(); b->pp_off.clear(); b->pp_n.clear();
        b->pair_mol.clear(); b->Q.clear(); b->fscale.clear(); b->f_local.clear(); b->pair_rec.clear();
        for (auto& l : b->class_list) l.clear();
        for (auto& l : b->class_seg) l.clear();
        b->P64 = PairTable<double>{}; b->P32 = PairTable<float>{}; b->Pdf = PairTable<df32>{};
        return st;
    }
    b->gpu_ready = true;
    return MESS_OK;
}

mess_status mess_derivative_basis(const mess_basis* b, mess_basis** out, std::vector<int>& raised,
                                  std::vector<int>& lowered)
{
    if (b->nmol != 1) { mess_set_error("derivative basis: single-molecule bases only"); return MESS_EINVAL; }
    std::vector<HostShell> sh(b->shells.begin(), b->shells.end());
    const int ns = (int)sh.size();
    raised.assign(ns, -1);
    lowered.assign(ns, -1);
    for (int k = 0; k < ns; ++k) {
        HostShell r = b->shells[k];
        if (r.l + 1 > MESS_LMAX) { mess_set_error("derivative basis: shells up to l = %d", MESS_LMAX - 1); return MESS_EINVAL; }
        r.l += 1;
        for (int i = 0; i < r.K; ++i) r.coef[i] = 2.0 * r.alpha[i] * b->shells[k].coef[i];
        raised[k] = (int)sh.size();
        sh.push_back(r);
    }
    for (int k = 0; k < ns; ++k) {
        if (b->shells[k].l == 0) continue;
        HostShell r = b->shells[k];
        r.l -= 1;
        lowered[k] = (int)sh.size();
        sh.push_back(r);
    }
    mess_basis* e = new (std::nothrow) mess_basis();
    if (!e) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    add_molecule(e, b->Z, b->xyz, sh);
    mess_status st = build_pairs(e);
    if (st == MESS_OK) st = build_schwarz(e);
    if (st != MESS_OK) { mess_free_basis(e); delete e; return st; }
    e->gpu_ready = true;
    *out = e;
    return MESS_OK;
}

mess_status mess_displaced_basis(const mess_basis* b, int atom, int axis, double dx, mess_basis** out)
{
    *out = nullptr;
    if (b->nmol != 1 || atom < 0 || atom >= b->natom || axis < 0 || axis > 2) {
        mess_set_error("displaced basis: bad arguments");
        return MESS_EINVAL;
    }
    mess_basis* d = new (std::nothrow) mess_basis();
    if (!d) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    std::vector<double> xyz(b->xyz);
    xyz[3 * atom + axis] += dx;
    std::vector<HostShell> sh(b->shells);
    for (HostShell& s : sh)
        if (s.atom == atom) s.R[axis] += dx;
    add_molecule(d, b->Z, xyz, sh);
    *out = d;
    return MESS_OK;
}

mess_status mess_atoms_basis(const mess_basis* b, std::vector<int>& elements, mess_basis** out)
{
    elements.clear();
    mess_basis* a = new (std::nothrow) mess_basis();
    if (!a) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    for (int at = 0; at < b->natom; ++at) {
        const int z = b->Z[at];
        if (std::find(elements.begin(), elements.end(), z) != elements.end()) continue;
        elements.push_back(z);
        std::vector<HostShell> sh;
        for (const HostShell& s : b->shells)
            if (s.atom == at) {
                HostShell c = s;
                c.atom = 0;
                c.R[0] = c.R[1] = c.R[2] = 0.0;
                sh.push_back(c);
            }
        add_molecule(a, std::vector<int>{z}, std::vector<double>{0.0, 0.0, 0.0}, sh);
    }
    mess_status st = build_pairs(a);
    if (st == MESS_OK) st = build_schwarz(a);
    if (st != MESS_OK) { mess_free_basis(a); delete a; return st; }
    a->gpu_ready = true;
    *out = a;
    return MESS_OK;
}

mess_status mess_batch_basis(int nmol, const mess_basis* const* bases, mess_basis** out)
{
    if (nmol <= 0 || !bases || !out) { mess_set_error("bad batch arguments"); return MESS_EINVAL; }
    mess_basis* b = new (std::nothrow) mess_basis();
    if (!b) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    for (int m = 0; m < nmol; ++m) {
        const mess_basis* s = bases[m];
        if (!s || s->nmol != 1) { delete b; mess_set_error("batch entry %d is not a single-molecule basis", m); return MESS_EINVAL; }
        add_molecule(b, s->Z, s->xyz, s->shells);
    }
    PhaseTimer tm(nullptr);
    mess_status st = build_pairs(b);
    tm.mark("batched basis: primitive pairs");
    if (st == MESS_OK) st = build_schwarz(b);
    tm.mark("batched basis: Schwarz factors");
    if (st != MESS_OK) { mess_free_basis(b); delete b; return st; }
    b->gpu_ready = true;
    *out = b;
    return MESS_OK;
}

extern "C" int mess_basis_nbf(const mess_basis* b) { return b ? b->nbf : -1; }
extern "C" int mess_basis_nshell(const mess_basis* b) { return b ? (int)b->shells.size() : -1; }
extern "C" int mess_basis_nelectron(const mess_basis* b) { return b ? b->nelec : -1; }

extern "C" void mess_basis_destroy(mess_basis* b)
{
    if (!b) return;
    mess_free_basis(b);
    delete b;
}

extern "C" double mess_nuclear_repulsion(const mess_basis* b)
{
    if (!b) return NAN;
    double e = 0.0;
    for (int a = 0; a < b->natom; ++a)
        for (int c = 0; c < a; ++c) {
            double r2 = 0.0;
            for (int x = 0; x < 3; ++x) { const double d = b->xyz[3 * a + x] - b->xyz[3 * c + x]; r2 += d * d; }
            e += (double)b->Z[a] * b->Z[c] / sqrt(r2);
        }
    return e;
}

extern "C" mess_status mess_schwarz(const mess_basis* b, double* Q)
{
    if (!b || !Q) { mess_set_error("null argument"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    const int ns = (int)b->shells.size();
    for (int i = 0; i < ns * ns; ++i) Q[i] = 0.0;
    for (int p = 0; p < b->npair; ++p) {
        Q[b->pair_a[p] * ns + b->pair_b[p]] = b->Q[p];
        Q[b->pair_b[p] * ns + b->pair_a[p]] = b->Q[p];
    }
    return MESS_OK;
}

// ------------------------------------------------------------------------------------------ one-electron
extern "C" mess_status mess_one_e_device(const mess_basis* b, double* dS, double* dT, double* dV, void* stream)
{
    if (!b) { mess_set_error("basis is NULL"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    MESS_CUDA_TRY(mess_launch_one_e(b, dS, dT, dV, (cudaStream_t)stream));
    return MESS_OK;
}

static mess_status one_e_host(const mess_basis* b, double* S, double* T, double* V)
{
    if (!b) { mess_set_error("basis is NULL"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    const size_t nn = (size_t)b->nbf * b->nbf;
    DevBuf<double> d;
    MESS_CUDA_TRY(d.alloc(nn));
    cudaError_t e = mess_launch_one_e(b, S ? d.p : nullptr, T ? d.p : nullptr, V ? d.p : nullptr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(S ? S : (T ? T : V), d.p, nn * sizeof(double), cudaMemcpyDeviceToHost);
    d.free();
    if (e != cudaSuccess) { mess_set_error("one-electron integrals: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}

extern "C" mess_status mess_overlap(const mess_basis* b, double* S)
{
    if (!S) { mess_set_error("S is NULL"); return MESS_EINVAL; }
    return one_e_host(b, S, nullptr, nullptr);
}
extern "C" mess_status mess_kinetic(const mess_basis* b, double* T)
{
    if (!T) { mess_set_error("T is NULL"); return MESS_EINVAL; }
    return one_e_host(b, nullptr, T, nullptr);
}
extern "C" mess_status mess_nuclear(const mess_basis* b, double* V)
{
    if (!V) { mess_set_error("V is NULL"); return MESS_EINVAL; }
    return one_e_host(b, nullptr, nullptr, V);
}

// ------------------------------------------------------------------------------------------ J / K
// Algorithmic flops of one primitive quartet / one shell quartet of a class (FMA = 2 flops):
// quartet set-up (exponent sums, P - Q, W - P, W - Q, T, prefactor) ~ 25, Boys (Taylor + exp +
// downward recursion) 18 + 3L, prefactor scaling L + 1, the VRR op count, the contraction adds;
// per shell quartet: the HRR op count and 6 FMAs per integral for the J/K digestion.
static void class_flops(int qc, double* per_prim, double* per_shell)
{
    const mess_qclass_info& c = MESS_QCLASS[qc];
    *per_prim = 25.0 + (18.0 + 3.0 * c.L) + (c.L + 1.0) + (double)c.vrr_flops + c.nacc;
    *per_shell = (double)c.hrr_flops + 12.0 * c.nint;
}

// kernel arithmetic of a part: the autotuner's choice, else FP64 / double-float for the split parts
// and FP32 (with or without FP64 Boys) for the others
static int part_mode(const BinPart& p, const mess_jk_opts& o)
{
    if (p.mode >= 0) return p.mode;
    if (p.fp64) return (o.prec == MESS_MIXED && o.split_df32) ? MESS_MODE_DF32 : MESS_MODE_FP64;
    return o.boys_fp64 ? MESS_MODE_MIXED : MESS_MODE_FP32;
}

// The launches of one J/K build, all on stream s or forked from it onto the pool's streams and
// joined back: zero J and K, convert D for the reduced-precision parts, one launch per bin part
// (most expensive first), symmetrise.  With parts != null every launch runs on s between timing
// events.  Used directly and under stream capture (the cached CUDA graph of a repeated build).
static mess_status jk_enqueue(mess_basis* b, const mess_jk_opts& o, const double* dD, double* dJ, double* dK,
                              cudaStream_t s, bool need32, bool needdf, StreamPool* pool,
                              std::vector<cudaEvent_t>* ev, mess_jk_info* info)
{
    const size_t bytes = (size_t)b->packed * sizeof(double);
    MESS_CUDA_TRY(cudaMemsetAsync(dJ, 0, bytes, s));
    MESS_CUDA_TRY(cudaMemsetAsync(dK, 0, bytes, s));
    mess_jk_info inf{};
    if (need32 || needdf) {
        MESS_CUDA_TRY(mess_launch_convert_density(dD, need32 ? b->d_D32.p : nullptr, needdf ? b->d_Ddf.p : nullptr,
                                                  b->packed, s));
        inf.kernel_launches += 1;
    }
    // launch order: most expensive parts first (FP64, then by algorithmic work)
    std::vector<size_t> order(b->bins.parts.size());
    std::iota(order.begin(), order.end(), (size_t)0);
    auto cost = [&](const BinPart& p) {
        double fp, fs;
        class_flops(p.qclass, &fp, &fs);
        return (fp * (double)p.prim_quartets + fs * (double)p.total) * (p.fp64 ? 62.0 : 1.0);
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return cost(b->bins.parts[x]) > cost(b->bins.parts[y]); });
    const bool concurrent = pool != nullptr;
    if (concurrent) {
        MESS_CUDA_TRY(cudaEventRecord(pool->fork, s));
        for (int i = 0; i < pool->n; ++i) MESS_CUDA_TRY(cudaStreamWaitEvent(pool->s[i], pool->fork, 0));
    }
    mess_status out = MESS_OK;
    for (size_t r = 0; r < order.size(); ++r) {
        const size_t k = order[r];
        const BinPart& p = b->bins.parts[k];
        ClassLaunchArgs a{};
        a.kind = MESS_KIND_JK;
        a.mode = part_mode(p, o);
        a.G = p.G;
        a.team = p.team;
        a.bin = bin_launch(b, p);
        a.P64_ptr = &b->P64;
        a.P32_ptr = &b->P32;
        a.Pdf_ptr = &b->Pdf;
        a.D = dD;
        a.D32 = b->d_D32.p;
        a.Ddf = b->d_Ddf.p;
        a.J = dJ;
        a.K = dK;
        a.n = b->nbf;
        a.stream = concurrent ? pool->s[r % pool->n] : s;
        if (ev) cudaEventRecord((*ev)[2 * k], s);
        cudaError_t e = MESS_CLASS_LAUNCHERS[p.qclass](a);
        if (ev) cudaEventRecord((*ev)[2 * k + 1], s);
        if (e != cudaSuccess) {
            mess_set_error("J/K kernel launch (class %d): %s", p.qclass, cudaGetErrorString(e));
            out = MESS_ECUDA;
            break;
        }
        inf.shell_quartets += p.total;
        inf.function_quartets += p.fn_quartets;
        inf.primitive_quartets += p.prim_quartets;
        if (p.fp64) inf.shell_quartets_fp64 += p.total;
        inf.kernel_launches += 1;
    }
    if (concurrent) {
        // join: s waits for every pool stream (also after a failed launch)
        for (int i = 0; i < pool->n; ++i) {
            cudaEventRecord(pool->join[i], pool->s[i]);
            cudaStreamWaitEvent(s, pool->join[i], 0);
        }
    }
    if (out == MESS_OK) {
        cudaError_t e = mess_launch_symmetrise_jk(b, dJ, dK, s);
        if (e != cudaSuccess) { mess_set_error("symmetrise: %s", cudaGetErrorString(e)); out = MESS_ECUDA; }
        inf.kernel_launches += 1;
    }
    *info = inf;
    return out;
}

void mess_free_jk_graphs(mess_basis* b)
{
    for (JKGraph& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// Capture the launches of one build into a graph on a private stream (thread-local capture mode,
// pool streams forked into the capture) and instantiate it.  Returns null if any step fails; the
// build then launches directly.
static cudaGraphExec_t jk_capture(mess_basis* b, const mess_jk_opts& o, const double* dD, double* dJ, double* dK,
                                  bool need32, bool needdf, StreamPool* pool, mess_jk_info* info)
{
    cudaStream_t cs = pool->capture;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
    mess_status st = jk_enqueue(b, o, dD, dJ, dK, cs, need32, needdf, b->bins.parts.size() > 1 ? pool : nullptr,
                                nullptr, info);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaGraphExec_t exec = nullptr;
    if (st == MESS_OK && e == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a failed capture leaves nothing sticky; clear the last-error slot
    return exec;
}

// The J/K options checked and reduced to what selects the quartet bins: screening threshold tau,
// split threshold tau64 (0 unless split == 2) and split (0: every quartet in FP64, 1: every quartet
// in FP32, 2: FP64-class above tau64 and FP32 below).  Shared by the builds and the bins query.
static mess_status jk_options(const mess_jk_opts* opts, mess_jk_opts* out, double* tau64_out, int* split_out)
{
    mess_jk_opts o{};
    if (opts) o = *opts;
    if (o.prec != MESS_FP64 && o.prec != MESS_MIXED && o.prec != MESS_FP32) {
        mess_set_error("unknown precision %d", (int)o.prec);
        return MESS_EINVAL;
    }
    if (!(o.schwarz_tau >= 0.0) || std::isnan(o.fp64_tau)) { mess_set_error("bad thresholds"); return MESS_EINVAL; }
    double tau64 = o.fp64_tau == 0.0 ? MESS_DEFAULT_FP64_TAU : o.fp64_tau;
    int split = 0;
    if (o.prec == MESS_MIXED) split = tau64 > 0.0 ? 2 : 1;
    else if (o.prec == MESS_FP32) split = 1;
    if (split != 2) tau64 = 0.0;
    *out = o;
    *tau64_out = tau64;
    *split_out = split;
    return MESS_OK;
}

// Argument checks shared by the J/K entry points, and the quartet bins for the options.
static mess_status jk_prepare(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts,
                              mess_jk_opts* out)
{
    if (!b || !dD || !dJ || !dK) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (dD == dJ || dD == dK || dJ == dK) { mess_set_error("D, J and K must be distinct buffers"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    double tau64 = 0.0;
    int split = 0;
    mess_status st = jk_options(opts, out, &tau64, &split);
    if (st != MESS_OK) return st;
    return mess_ensure_bins(b, out->schwarz_tau, tau64, split);
}

static mess_status jk_run(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts,
                          mess_jk_info* info, mess_jk_part* parts, int max_parts, int* nparts, bool graphs = true)
{
    mess_jk_opts o{};
    mess_status st = jk_prepare(b, dD, dJ, dK, opts, &o);
    if (st != MESS_OK) return st;
    if (parts && (int)b->bins.parts.size() > max_parts) {
        mess_set_error("mess_jk_profile: %d launches, max_parts = %d", (int)b->bins.parts.size(), max_parts);
        return MESS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    // FP32 / double-float copies of D for the reduced-precision parts, made once per build; the
    // previous build on this basis must be done with them first
    bool need32 = false, needdf = false;
    for (const BinPart& p : b->bins.parts) {
        const int m = part_mode(p, o);
        if (m == MESS_MODE_FP32 || m == MESS_MODE_MIXED) need32 = true;
        else if (m == MESS_MODE_DF32) needdf = true;
    }
    if ((need32 && !b->d_D32.p) || (needdf && !b->d_Ddf.p) || ((need32 || needdf) && !b->dconv_free)) {
        mess_set_error("density copies missing");
        return MESS_ECUDA;
    }
    if (need32 || needdf) MESS_CUDA_TRY(cudaStreamWaitEvent(s, b->dconv_free, 0));
    mess_jk_info inf{};
    mess_status out = MESS_OK;
    if (parts) {
        std::vector<cudaEvent_t> ev(2 * b->bins.parts.size());
        for (auto& e : ev) MESS_CUDA_TRY(cudaEventCreate(&e));
        out = jk_enqueue(b, o, dD, dJ, dK, s, need32, needdf, nullptr, &ev, &inf);
        if (out == MESS_OK) {
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { mess_set_error("profile sync: %s", cudaGetErrorString(e)); out = MESS_ECUDA; }
        }
        for (size_t k = 0; out == MESS_OK && k < b->bins.parts.size(); ++k) {
            const BinPart& p = b->bins.parts[k];
            const mess_qclass_info& c = MESS_QCLASS[p.qclass];
            mess_jk_part& r = parts[k];
            r.qclass = p.qclass;
            r.la = c.la; r.lb = c.lb; r.lc = c.lc; r.ld = c.ld;
            r.fp64 = p.fp64;
            r.shell_quartets = p.total;
            r.primitive_quartets = p.prim_quartets;
            r.function_quartets = p.fn_quartets;
            r.G = p.G;
            r.team = p.team;
            r.mode = part_mode(p, o);
            double fp, fs;
            class_flops(p.qclass, &fp, &fs);
            r.flops = fp * (double)p.prim_quartets + fs * (double)p.total;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
            r.ms = ms;
        }
        if (out == MESS_OK && nparts) *nparts = (int)b->bins.parts.size();
        for (auto& e : ev) cudaEventDestroy(e);
    } else {
        StreamPool* pool = nullptr;
        MESS_CUDA_TRY(get_pool(&pool));
        std::unique_lock<std::mutex> lk(pool->mu);
        // A build repeated with the same buffers, options and bins (an SCF loop, a benchmark) runs
        // as one CUDA graph launch instead of one launch per part: captured on the second such call,
        // replayed from the third.  Not while the caller's stream is itself being captured.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        MESS_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
        JKGraph* g = nullptr;
        if (graphs && cap == cudaStreamCaptureStatusNone) {
            for (JKGraph& x : b->graphs)
                if (x.bins_gen == b->bins.generation && x.prec == o.prec && x.boys_fp64 == o.boys_fp64 &&
                    x.split_df32 == o.split_df32 && x.D == dD && x.J == dJ && x.K == dK) g = &x;
            if (!g) {
                if (b->graphs.size() >= 4) {
                    if (b->graphs.front().exec) cudaGraphExecDestroy(b->graphs.front().exec);
                    b->graphs.erase(b->graphs.begin());
                }
                JKGraph x{};
                x.bins_gen = b->bins.generation;
                x.prec = o.prec; x.boys_fp64 = o.boys_fp64; x.split_df32 = o.split_df32;
                x.D = dD; x.J = dJ; x.K = dK;
                b->graphs.push_back(x);
            } else if (!g->exec && !g->failed) {
                g->exec = jk_capture(b, o, dD, dJ, dK, need32, needdf, pool, &g->info);
                if (!g->exec) g->failed = 1;
            }
        }
        if (g && g->exec) {
            MESS_CUDA_TRY(cudaGraphLaunch(g->exec, s));
            inf = g->info;
        } else {
            out = jk_enqueue(b, o, dD, dJ, dK, s, need32, needdf, b->bins.parts.size() > 1 ? pool : nullptr, nullptr,
                             &inf);
        }
    }
    if (need32 || needdf) cudaEventRecord(b->dconv_free, s);
    if (info) *info = inf;
    return out;
}

extern "C" mess_status mess_jk_build_device(const mess_basis* bc, const double* dD, double* dJ, double* dK,
                                            const mess_jk_opts* opts, mess_jk_info* info)
{
    return jk_run(const_cast<mess_basis*>(bc), dD, dJ, dK, opts, info, nullptr, 0, nullptr);
}

mess_status mess_jk_packed(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts,
                           mess_jk_info* info, bool graphs)
{
    return jk_run(b, dD, dJ, dK, opts, info, nullptr, 0, nullptr, graphs);
}

mess_status mess_jk_ensure_bins(mess_basis* b, const mess_jk_opts* opts)
{
    static double dummy[3];
    mess_jk_opts o{};
    return jk_prepare(b, dummy, dummy + 1, dummy + 2, opts, &o);
}

mess_status mess_jk_enqueue_only(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts)
{
    mess_jk_opts o{};
    double tau64 = 0.0;
    int split = 0;
    mess_status st = jk_options(opts, &o, &tau64, &split);
    if (st != MESS_OK) return st;
    const BinSet& B = b->bins;
    if (!(B.tau == o.schwarz_tau && B.tau64 == tau64 && B.split == split && B.active_version == b->active_version)) {
        mess_set_error("J/K enqueue: the quartet bins for these options are not built");
        return MESS_EINVAL;
    }
    bool need32 = false, needdf = false;
    for (const BinPart& p : b->bins.parts) {
        const int m = part_mode(p, o);
        if (m == MESS_MODE_FP32 || m == MESS_MODE_MIXED) need32 = true;
        else if (m == MESS_MODE_DF32) needdf = true;
    }
    if ((need32 && !b->d_D32.p) || (needdf && !b->d_Ddf.p)) { mess_set_error("density copies missing"); return MESS_ECUDA; }
    StreamPool* pool = nullptr;
    MESS_CUDA_TRY(get_pool(&pool));
    std::unique_lock<std::mutex> lk(pool->mu);
    mess_jk_info inf{};
    return jk_enqueue(b, o, dD, dJ, dK, (cudaStream_t)o.cuda_stream, need32, needdf,
                      b->bins.parts.size() > 1 ? pool : nullptr, nullptr, &inf);
}

mess_status mess_jk_bins_ready(const mess_basis* b, const mess_jk_opts* opts, bool* ready)
{
    mess_jk_opts o{};
    double tau64 = 0.0;
    int split = 0;
    mess_status st = jk_options(opts, &o, &tau64, &split);
    if (st != MESS_OK) return st;
    const BinSet& B = b->bins;
    *ready = B.tau == o.schwarz_tau && B.tau64 == tau64 && B.split == split && B.active_version == b->active_version;
    return MESS_OK;
}

extern "C" mess_status mess_jk_profile(const mess_basis* bc, const double* dD, double* dJ, double* dK,
                                       const mess_jk_opts* opts, mess_jk_part* parts, int max_parts, int* nparts)
{
    if (!parts || !nparts || max_parts <= 0) { mess_set_error("mess_jk_profile: no output array"); return MESS_EINVAL; }
    return jk_run(const_cast<mess_basis*>(bc), dD, dJ, dK, opts, nullptr, parts, max_parts, nparts);
}

// Autotuner: for every part of the bins, time each kernel variant that computes it (several copies
// at once, see below) - lanes per
// quartet G in {1, 4, 8, 32} (straight-line classes), one warp or one block of MESS_TEAM_WARPS warps per
// quartet, or a block whose warps split the quartet's primitive loop (classes with those kernels),
// and for the split parts FP64 or double-float arithmetic (when the options allow double-float) -
// alone on the stream, and keep the fastest.  The choice lives with the bins (a rebuild of the
// bins for other options starts from the fixed rules again).
static mess_status jk_autotune_device(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts,
                                      int reps, int* nchanged)
{
    mess_jk_opts o{};
    mess_status st = jk_prepare(b, dD, dJ, dK, opts, &o);
    if (st != MESS_OK) return st;
    if (reps < 1) reps = 1;
    if (reps > 50) reps = 50;
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    if (b->dconv_free) MESS_CUDA_TRY(cudaStreamWaitEvent(s, b->dconv_free, 0));
    MESS_CUDA_TRY(mess_launch_convert_density(dD, b->d_D32.p, b->d_Ddf.p, b->packed, s));
    StreamPool* pool = nullptr;
    MESS_CUDA_TRY(get_pool(&pool));
    std::unique_lock<std::mutex> lk(pool->mu);
    cudaEvent_t e0, e1;
    MESS_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); mess_set_error("%s", cudaGetErrorString(ce)); return MESS_ECUDA; }
    struct Variant { int G, team, mode; };
    int changed = 0;
    mess_status out = MESS_OK;
    for (BinPart& p : b->bins.parts) {
        const mess_qclass_info& c = MESS_QCLASS[p.qclass];
        std::vector<int> modes;
        if (p.fp64) {
            modes.push_back(MESS_MODE_FP64);
            if (o.prec == MESS_MIXED && o.split_df32 && b->d_Ddf.p) modes.push_back(MESS_MODE_DF32);
        } else {
            modes.push_back(o.boys_fp64 ? MESS_MODE_MIXED : MESS_MODE_FP32);
        }
        std::vector<Variant> cand;
        for (int m : modes) {
            if (c.straight) {
                cand.push_back({1, 0, m});
                cand.push_back({4, 0, m});
                cand.push_back({8, 0, m});
                cand.push_back({32, 0, m});
            } else {
                cand.push_back({1, 0, m});
            }
            if (c.team) {
                cand.push_back({1, 1, m});
                cand.push_back({1, 2, m});
                cand.push_back({1, 3, m});
            }
        }
        const Variant before{p.G, p.team, part_mode(p, o)};
        Variant best = before;
        float best_ms = 3.4e38f;
        for (const Variant& v : cand) {
            ClassLaunchArgs a{};
            a.kind = MESS_KIND_JK;
            a.mode = v.mode;
            a.G = v.G;
            a.team = v.team;
            a.bin = bin_launch(b, p);
            a.P64_ptr = &b->P64;
            a.P32_ptr = &b->P32;
            a.Pdf_ptr = &b->Pdf;
            a.D = dD;
            a.D32 = b->d_D32.p;
            a.Ddf = b->d_Ddf.p;
            a.J = dJ;
            a.K = dK;
            a.n = b->nbf;
            a.stream = s;
            // one untimed launch (first use of a kernel loads it), then the minimum over reps of the
            // time for MESS_TUNE_COPIES copies launched together on the pool's streams: the parts of
            // a build run concurrently, so a variant is charged for the GPU it occupies as well as
            // for its latency (a lane split that only fills idle SMs costs nothing extra; one that
            // crowds out the other parts does)
            a.stream = s;
            cudaError_t e = MESS_CLASS_LAUNCHERS[p.qclass](a);
            float vmin = 3.4e38f;
            for (int r = 0; e == cudaSuccess && r < reps; ++r) {
                cudaEventRecord(e0, s);
                cudaEventRecord(pool->fork, s);
                for (int c = 0; e == cudaSuccess && c < MESS_TUNE_COPIES; ++c) {
                    cudaStreamWaitEvent(pool->s[c], pool->fork, 0);
                    a.stream = pool->s[c];
                    e = MESS_CLASS_LAUNCHERS[p.qclass](a);
                    cudaEventRecord(pool->join[c], pool->s[c]);
                    cudaStreamWaitEvent(s, pool->join[c], 0);
                }
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess) vmin = std::min(vmin, ms);
            }
            if (e != cudaSuccess) {
                mess_set_error("autotune launch (class %d): %s", p.qclass, cudaGetErrorString(e));
                out = MESS_ECUDA;
                break;
            }
            if (vmin < best_ms) { best_ms = vmin; best = v; }
        }
        if (out != MESS_OK) break;
        if (best.G != before.G || best.team != before.team || best.mode != before.mode) ++changed;
        p.G = best.G;
        p.team = best.team;
        p.mode = best.mode;
        p.tuned = 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // kernels changed: cached graphs of these bins are stale
    b->bins.generation += 1;
    mess_free_jk_graphs(b);
    if (b->dconv_free) cudaEventRecord(b->dconv_free, s);
    if (nchanged) *nchanged = changed;
    return out;
}

extern "C" mess_status mess_jk_set_variant(const mess_basis* bc, const mess_jk_opts* opts, int G, int team,
                                           int split_mode, int* nchanged)
{
    if (!bc) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (G != 1 && G != 4 && G != 8 && G != 32) { mess_set_error("G must be 1, 4, 8 or 32"); return MESS_EINVAL; }
    if (team < 0 || team > 3) { mess_set_error("team must be 0, 1, 2 or 3"); return MESS_EINVAL; }
    if (split_mode != -1 && split_mode != MESS_MODE_FP64 && split_mode != MESS_MODE_DF32) {
        mess_set_error("split_mode must be -1, 0 (FP64) or 3 (double-float)");
        return MESS_EINVAL;
    }
    mess_basis* b = const_cast<mess_basis*>(bc);
    mess_jk_opts o{};
    // jk_prepare wants distinct buffer pointers; none is touched here
    static double dummy[3];
    mess_status st = jk_prepare(b, dummy, dummy + 1, dummy + 2, opts, &o);
    if (st != MESS_OK) return st;
    if (split_mode == MESS_MODE_DF32 && !(o.prec == MESS_MIXED && o.split_df32)) {
        mess_set_error("double-float split parts need prec MESS_MIXED with split_df32");
        return MESS_EINVAL;
    }
    int changed = 0;
    for (BinPart& p : b->bins.parts) {
        const mess_qclass_info& c = MESS_QCLASS[p.qclass];
        const int G0 = p.G, t0 = p.team, m0 = part_mode(p, o);
        if (!c.straight) { p.G = 1; p.team = team; }                  // op-program classes: G = 1 only
        else if (team && c.team) { p.team = team; p.G = 1; }
        else { p.team = 0; p.G = G; }
        if (p.fp64 && split_mode >= 0) p.mode = split_mode;
        if (p.G != G0 || p.team != t0 || part_mode(p, o) != m0) ++changed;
    }
    b->bins.generation += 1;
    mess_free_jk_graphs(b);
    if (nchanged) *nchanged = changed;
    return MESS_OK;
}

// The kernel choice of every part of the bins for these options, as 4 ints per part: quartet class,
// G, team, arithmetic (MESS_MODE_*).  Saved by one process (after autotuning) and restored by another
// (for instance a profiling run, whose own timings would be distorted by the profiler).
extern "C" mess_status mess_jk_get_tuning(const mess_basis* bc, const mess_jk_opts* opts, int* table, int max_parts,
                                          int* nparts)
{
    if (!bc || !nparts) { mess_set_error("null argument"); return MESS_EINVAL; }
    mess_basis* b = const_cast<mess_basis*>(bc);
    mess_jk_opts o{};
    static double dummy[3];
    mess_status st = jk_prepare(b, dummy, dummy + 1, dummy + 2, opts, &o);
    if (st != MESS_OK) return st;
    const int np = (int)b->bins.parts.size();
    *nparts = np;
    if (!table) return MESS_OK;
    if (max_parts < np) { mess_set_error("mess_jk_get_tuning: %d parts, max_parts = %d", np, max_parts); return MESS_EINVAL; }
    for (int k = 0; k < np; ++k) {
        const BinPart& p = b->bins.parts[k];
        table[4 * k] = p.qclass;
        table[4 * k + 1] = p.G;
        table[4 * k + 2] = p.team;
        table[4 * k + 3] = part_mode(p, o);
    }
    return MESS_OK;
}

extern "C" mess_status mess_jk_set_tuning(const mess_basis* bc, const mess_jk_opts* opts, const int* table, int nparts)
{
    if (!bc || !table) { mess_set_error("null argument"); return MESS_EINVAL; }
    mess_basis* b = const_cast<mess_basis*>(bc);
    mess_jk_opts o{};
    static double dummy[3];
    mess_status st = jk_prepare(b, dummy, dummy + 1, dummy + 2, opts, &o);
    if (st != MESS_OK) return st;
    if (nparts != (int)b->bins.parts.size()) {
        mess_set_error("mess_jk_set_tuning: %d entries for %d parts", nparts, (int)b->bins.parts.size());
        return MESS_EINVAL;
    }
    // validate everything before changing anything
    for (int k = 0; k < nparts; ++k) {
        const BinPart& p = b->bins.parts[k];
        const mess_qclass_info& c = MESS_QCLASS[p.qclass];
        const int qc = table[4 * k], G = table[4 * k + 1], team = table[4 * k + 2], mode = table[4 * k + 3];
        bool ok = qc == p.qclass && team >= 0 && team <= 3 && (team == 0 || c.team);
        ok = ok && (team ? G == 1 : (c.straight ? (G == 1 || G == 4 || G == 8 || G == 32) : G == 1));
        if (p.fp64) ok = ok && (mode == MESS_MODE_FP64 || (mode == MESS_MODE_DF32 && o.prec == MESS_MIXED && o.split_df32));
        else ok = ok && mode == (o.boys_fp64 ? MESS_MODE_MIXED : MESS_MODE_FP32);
        if (!ok) { mess_set_error("mess_jk_set_tuning: entry %d does not fit part %d", k, k); return MESS_EINVAL; }
    }
    for (int k = 0; k < nparts; ++k) {
        BinPart& p = b->bins.parts[k];
        p.G = table[4 * k + 1];
        p.team = table[4 * k + 2];
        p.mode = table[4 * k + 3];
        p.tuned = 1;
    }
    b->bins.generation += 1;
    mess_free_jk_graphs(b);
    return MESS_OK;
}

extern "C" mess_status mess_jk_autotune(const mess_basis* bc, const double* D, const mess_jk_opts* opts, int reps,
                                        int* nchanged)
{
    if (!bc || !D) { mess_set_error("null argument"); return MESS_EINVAL; }
    mess_basis* b = const_cast<mess_basis*>(bc);
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    if (b->nmol != 1) { mess_set_error("mess_jk_autotune: single-molecule bases only"); return MESS_EINVAL; }
    const size_t nn = (size_t)b->nbf * b->nbf;
    DevBuf<double> d;
    MESS_CUDA_TRY(d.alloc(3 * nn));
    mess_jk_opts o{};
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    mess_status st = MESS_OK;
    cudaError_t e = cudaMemcpyAsync(d.p, D, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = jk_autotune_device(b, d.p, d.p + nn, d.p + 2 * nn, &o, reps, nchanged);
        e = cudaStreamSynchronize(s);
    }
    d.free();
    if (st != MESS_OK) return st;
    if (e != cudaSuccess) { mess_set_error("jk_autotune: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}

extern "C" mess_status mess_jk_build(const mess_basis* bc, const double* D, double* J, double* K,
                                     const mess_jk_opts* opts, mess_jk_info* info)
{
    if (!bc || !D || !J || !K) { mess_set_error("null argument"); return MESS_EINVAL; }
    mess_basis* b = const_cast<mess_basis*>(bc);
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    const size_t nn = (size_t)b->nbf * b->nbf;
    // D, J, K staged in a device buffer kept with the basis (allocated by the first call): repeated
    // calls allocate nothing, and their builds replay as one CUDA graph
    if (b->d_stage.n < 3 * nn) MESS_CUDA_TRY(b->d_stage.alloc(3 * nn));
    double* d = b->d_stage.p;
    mess_jk_opts o{};
    if (opts) o = *opts;
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    mess_status st = MESS_OK;
    cudaError_t e = cudaMemcpyAsync(d, D, nn * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        st = mess_jk_build_device(b, d, d + nn, d + 2 * nn, &o, info);
        if (st == MESS_OK) {
            e = cudaMemcpyAsync(J, d + nn, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(K, d + 2 * nn, nn * sizeof(double), cudaMemcpyDeviceToHost, s);
        }
    }
    // the staging buffer is free again only once the stream has drained
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    if (st != MESS_OK) return st;
    if (e != cudaSuccess) { mess_set_error("jk_build: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}

extern "C" mess_status mess_eri_tensor(const mess_basis* bc, double* G)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !G) { mess_set_error("null argument"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    const int n = b->nbf;
    if (n > 64) { mess_set_error("mess_eri_tensor: n = %d > 64", n); return MESS_EINVAL; }
    mess_status st = mess_ensure_bins(b, 0.0, 0.0, 0);
    if (st != MESS_OK) return st;
    const size_t n4 = (size_t)n * n * n * n;
    DevBuf<double> d;
    MESS_CUDA_TRY(d.alloc(n4));
    cudaError_t e = cudaMemset(d.p, 0, n4 * sizeof(double));
    for (const BinPart& p : b->bins.parts) {
        if (e != cudaSuccess) break;
        ClassLaunchArgs a{};
        a.kind = MESS_KIND_STORE;
        a.bin = bin_launch(b, p);
        a.P64_ptr = &b->P64;
        a.P32_ptr = &b->P32;
        a.out = d.p;
        a.n = n;
        e = MESS_CLASS_LAUNCHERS[p.qclass](a);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(G, d.p, n4 * sizeof(double), cudaMemcpyDeviceToHost);
    d.free();
    if (e != cudaSuccess) { mess_set_error("eri_tensor: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}

extern "C" mess_status mess_profiler_range(int on)
{
    const cudaError_t e = on ? cudaProfilerStart() : cudaProfilerStop();
    if (e != cudaSuccess) { mess_set_error("profiler range: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}
