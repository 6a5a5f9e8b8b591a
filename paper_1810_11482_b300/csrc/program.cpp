// Run-time compiled user programs (the paper's `program`, Sec. 4 and
// Listing 2: create_program_with_file, build(kernel name) returning a
// future, run(args, name, grid, block) returning a future).
//
// Compilation uses NVRTC (loaded with dlopen on first use, so the library
// loads without it) for the device's own architecture; the CUBIN is loaded
// with cudaLibraryLoadData and kernels are launched as cudaKernel_t through
// cudaLaunchKernel on the program's device and stream slot.  A build runs
// on the worker pool; every run of the program depends on its last build.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <sstream>

#include "runtime.hpp"

using namespace hxc;

namespace {

constexpr uint32_t kProgMagic = 0x9506A301u;

struct Nvrtc {
    bool ok = false;
    std::string why;
    nvrtcResult (*create)(nvrtcProgram *, const char *, const char *, int, const char *const *,
                          const char *const *) = nullptr;
    nvrtcResult (*compile)(nvrtcProgram, int, const char *const *) = nullptr;
    nvrtcResult (*log_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*log)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t *) = nullptr;
    nvrtcResult (*cubin)(nvrtcProgram, char *) = nullptr;
    nvrtcResult (*add_name)(nvrtcProgram, const char *) = nullptr;
    nvrtcResult (*lowered)(nvrtcProgram, const char *, const char **) = nullptr;
    nvrtcResult (*destroy)(nvrtcProgram *) = nullptr;
    const char *(*errstr)(nvrtcResult) = nullptr;
};

Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"};
        void *h = nullptr;
        for (const char *nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            n.why = "NVRTC (libnvrtc.so.13) not found";
            return;
        }
#define SYM(field, name) n.field = reinterpret_cast<decltype(n.field)>(dlsym(h, name))
        SYM(create, "nvrtcCreateProgram");
        SYM(compile, "nvrtcCompileProgram");
        SYM(log_size, "nvrtcGetProgramLogSize");
        SYM(log, "nvrtcGetProgramLog");
        SYM(cubin_size, "nvrtcGetCUBINSize");
        SYM(cubin, "nvrtcGetCUBIN");
        SYM(add_name, "nvrtcAddNameExpression");
        SYM(lowered, "nvrtcGetLoweredName");
        SYM(destroy, "nvrtcDestroyProgram");
        SYM(errstr, "nvrtcGetErrorString");
#undef SYM
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin &&
               n.add_name && n.lowered && n.destroy && n.errstr;
        if (!n.ok) n.why = "NVRTC symbols missing";
    });
    return n;
}

struct Program : RefCounted {
    uint32_t magic = kProgMagic;
    Ref<Device> dev;
    std::string source, name;
    std::mutex m;
    std::vector<cudaLibrary_t> libs;  // every build's library, kept until the program dies
    std::map<std::string, cudaKernel_t> kernels;  // by requested name
    std::string log;
    FutRef built;  // last build (runs depend on it)
    ~Program() override {
        for (auto l : libs) cudaLibraryUnload(l);
    }
};

Ref<Program> prog_from_handle(hxc_program h) {
    Program *p = reinterpret_cast<Program *>(h);
    if (!p || p->magic != kProgMagic) {
        set_error("invalid program handle");
        return Ref<Program>();
    }
    return Ref<Program>(p, false);
}

std::vector<std::string> split_list(const char *s, char sep) {
    std::vector<std::string> out;
    if (!s) return out;
    std::string cur;
    for (const char *c = s;; c++) {
        if (*c == sep || *c == 0) {
            size_t a = cur.find_first_not_of(" \t\n"), b = cur.find_last_not_of(" \t\n");
            if (a != std::string::npos) out.push_back(cur.substr(a, b - a + 1));
            cur.clear();
            if (!*c) break;
        } else {
            cur.push_back(*c);
        }
    }
    return out;
}

// Compiles and loads; returns the status stored in the build future.
hxc_status do_build(Program *p, const std::vector<std::string> &names,
                    const std::vector<std::string> &opts) {
    Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        std::lock_guard<std::mutex> g(p->m);
        p->log = nv.why;
        return HXC_E_UNSUPPORTED;
    }
    nvrtcProgram prog;
    if (nv.create(&prog, p->source.c_str(), p->name.c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        std::lock_guard<std::mutex> g(p->m);
        p->log = "nvrtcCreateProgram failed";
        return HXC_E_INVALID;
    }
    for (auto &n : names) nv.add_name(prog, n.c_str());
    char arch[64];
    snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%d", p->dev->prop.major, p->dev->prop.minor);
    std::vector<std::string> all{arch, "-std=c++17"};
    for (auto &o : opts) all.push_back(o);
    std::vector<const char *> av;
    for (auto &o : all) av.push_back(o.c_str());
    nvrtcResult r = nv.compile(prog, (int)av.size(), av.data());
    size_t ls = 0;
    nv.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) nv.log(prog, &log[0]);
    while (!log.empty() && log.back() == '\0') log.pop_back();
    {
        std::lock_guard<std::mutex> g(p->m);
        p->log = log;
    }
    if (r != NVRTC_SUCCESS) {
        nv.destroy(&prog);
        return HXC_E_INVALID;
    }
    std::vector<std::string> lowered;
    for (auto &n : names) {
        const char *lw = nullptr;
        if (nv.lowered(prog, n.c_str(), &lw) != NVRTC_SUCCESS || !lw) {
            nv.destroy(&prog);
            std::lock_guard<std::mutex> g(p->m);
            p->log += "\nkernel '" + n + "' not found in the program";
            return HXC_E_INVALID;
        }
        lowered.push_back(lw);
    }
    size_t cs = 0;
    nv.cubin_size(prog, &cs);
    std::string cubin(cs, '\0');
    nv.cubin(prog, &cubin[0]);
    nv.destroy(&prog);
    hxc_status st = p->dev->make_current();
    if (st) return st;
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return cuda_status(e, "cudaLibraryLoadData");
    std::map<std::string, cudaKernel_t> ks;
    for (size_t i = 0; i < names.size(); i++) {
        cudaKernel_t k = nullptr;
        e = cudaLibraryGetKernel(&k, lib, lowered[i].c_str());
        if (e != cudaSuccess) {
            cudaLibraryUnload(lib);
            return cuda_status(e, "cudaLibraryGetKernel");
        }
        ks[names[i]] = k;
    }
    std::lock_guard<std::mutex> g(p->m);
    p->libs.push_back(lib);
    for (auto &kv : ks) p->kernels[kv.first] = kv.second;
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_program_create_with_source(hxc_device dh, const char *source, const char *name,
                                          hxc_program *out) {
    if (!out || !source) {
        set_error("hxc_program_create_with_source: NULL argument");
        return HXC_E_INVALID;
    }
    Ref<Device> d = dev_from_handle(dh);
    if (!d) return HXC_E_INVALID;
    Program *p = new Program();
    p->dev = d;
    p->source = source;
    p->name = name ? name : "program.cu";
    *out = reinterpret_cast<hxc_program>(p);
    return HXC_OK;
}

hxc_status hxc_program_create_with_file(hxc_device dh, const char *path, hxc_program *out) {
    if (!path) {
        set_error("hxc_program_create_with_file: NULL path");
        return HXC_E_INVALID;
    }
    std::ifstream f(path, std::ios::binary);
    if (!f) {
        set_error("hxc_program_create_with_file: cannot read %s", path);
        return HXC_E_INVALID;
    }
    std::stringstream ss;
    ss << f.rdbuf();
    std::string src = ss.str();
    const char *slash = strrchr(path, '/');
    return hxc_program_create_with_source(dh, src.c_str(), slash ? slash + 1 : path, out);
}

hxc_status hxc_program_build(hxc_program ph, const char *kernel_names, const char *options,
                             const hxc_future *deps, int ndeps, hxc_future *out) {
    if (!out) {
        set_error("hxc_program_build: NULL output");
        return HXC_E_INVALID;
    }
    Ref<Program> p = prog_from_handle(ph);
    if (!p) return HXC_E_INVALID;
    std::vector<std::string> names = split_list(kernel_names, ',');
    if (names.empty()) {
        set_error("hxc_program_build: no kernel name");
        return HXC_E_INVALID;
    }
    std::vector<std::string> opts = split_list(options, ' ');
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    FutRef r = make_pending();
    auto go = [p, names, opts, r]() {
        pool().submit([p, names, opts, r] { fut_set_done(r, do_build(p.get(), names, opts)); });
    };
    if (dv.empty()) {
        go();
    } else {
        struct J {
            std::atomic<int> left{0};
            std::atomic<int> failed{0};
        };
        auto j = std::make_shared<J>();
        j->left = (int)dv.size();
        for (auto &f : dv)
            fut_on_done(f, [j, go, r](hxc_status s) {
                if (s != HXC_OK) j->failed = 1;
                if (j->left.fetch_sub(1) == 1) {
                    if (j->failed)
                        fut_set_done(r, HXC_E_DEP_FAILED);
                    else
                        go();
                }
            });
    }
    {
        std::lock_guard<std::mutex> g(p->m);
        p->built = r;
    }
    *out = to_handle(r);
    return HXC_OK;
}

hxc_status hxc_program_build_log(hxc_program ph, char *buf, size_t cap, size_t *len) {
    Ref<Program> p = prog_from_handle(ph);
    if (!p) return HXC_E_INVALID;
    std::lock_guard<std::mutex> g(p->m);
    if (len) *len = p->log.size();
    if (buf && cap) {
        size_t n = std::min(cap - 1, p->log.size());
        memcpy(buf, p->log.data(), n);
        buf[n] = 0;
    }
    return HXC_OK;
}

hxc_status hxc_program_run(hxc_program ph, const char *kernel_name, const hxc_kernel_arg *args,
                           int nargs, const hxc_launch_cfg *cfg, int slot, const hxc_future *deps,
                           int ndeps, hxc_future *out) {
    if (!out || !kernel_name || !cfg || nargs < 0 || (nargs && !args)) {
        set_error("hxc_program_run: NULL or invalid argument");
        return HXC_E_INVALID;
    }
    Ref<Program> p = prog_from_handle(ph);
    if (!p) return HXC_E_INVALID;
    const uint64_t g = (uint64_t)cfg->grid[0] * cfg->grid[1] * cfg->grid[2];
    const uint64_t b = (uint64_t)cfg->block[0] * cfg->block[1] * cfg->block[2];
    if (g == 0 || b == 0 || b > 1024) {
        set_error("hxc_program_run: empty grid or block > 1024 threads");
        return HXC_E_INVALID;
    }
    // kernel parameters: buffers become their device pointers, values are
    // copied now (the caller's memory may change before the launch)
    struct Params {
        std::vector<std::vector<unsigned char>> store;
        std::vector<void *> ptrs;
    };
    auto prm = std::make_shared<Params>();
    std::vector<AnyRef> keep;
    prm->store.resize(nargs);
    for (int i = 0; i < nargs; i++) {
        if (args[i].buf) {
            Ref<Buffer> bf = buf_from_handle(args[i].buf);
            if (!bf) return HXC_E_INVALID;
            if (bf->dev.get() != p->dev.get()) {
                set_error("hxc_program_run: argument %d lives on another device", i);
                return HXC_E_INVALID;
            }
            prm->store[i].resize(sizeof(void *));
            memcpy(prm->store[i].data(), &bf->ptr, sizeof(void *));
            keep.push_back(AnyRef(bf.get(), false));
        } else {
            if (!args[i].value || args[i].size == 0 || args[i].size > 4096) {
                set_error("hxc_program_run: argument %d has no buffer and no value", i);
                return HXC_E_INVALID;
            }
            prm->store[i].assign(static_cast<const unsigned char *>(args[i].value),
                                 static_cast<const unsigned char *>(args[i].value) + args[i].size);
        }
    }
    for (auto &s : prm->store) prm->ptrs.push_back(s.data());
    std::vector<FutRef> dv;
    hxc_status st = deps_from_handles(deps, ndeps, &dv);
    if (st) return st;
    {
        std::lock_guard<std::mutex> gl(p->m);
        if (p->built) dv.push_back(p->built);  // runs follow the program's last build
    }
    std::string name = kernel_name;
    Ref<Program> pr = p;
    dim3 grid(cfg->grid[0], cfg->grid[1], cfg->grid[2]), block(cfg->block[0], cfg->block[1], cfg->block[2]);
    keep.push_back(AnyRef(p.get(), false));
    StreamOp op = [pr, name, prm, grid, block](cudaStream_t s) -> cudaError_t {
        cudaKernel_t k = nullptr;
        {
            std::lock_guard<std::mutex> gl(pr->m);
            auto it = pr->kernels.find(name);
            if (it != pr->kernels.end()) k = it->second;
        }
        if (!k) return cudaErrorInvalidDeviceFunction;  // not built (or build failed)
        return cudaLaunchKernel(reinterpret_cast<const void *>(k), grid, block, prm->ptrs.data(), 0, s);
    };
    FutRef f;
    if ((st = issue_device_op(p->dev.get(), slot, dv, std::move(op), std::move(keep), &f))) return st;
    *out = to_handle(f);
    return HXC_OK;
}

hxc_status hxc_program_release(hxc_program ph) {
    Program *p = reinterpret_cast<Program *>(ph);
    if (!p || p->magic != kProgMagic) {
        set_error("invalid program handle");
        return HXC_E_INVALID;
    }
    p->release();
    return HXC_OK;
}

}  // extern "C"
