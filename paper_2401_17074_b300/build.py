"""Build step of the TSLB CUDA library, in-tree, for sm_103a.

Two variants of the same sources:
  libtslb.so          the product library;
  libtslb_checked.so  -DTSLB_CHECKED: every kernel tests its global-memory
                      indices and, on one out of range, records bit 4 of the
                      device status word and skips the access instead of
                      faulting (the stand-in for a memory checker; selected at
                      load time with TSLB_CHECKED=1).
Each source compiles to an object under _build/ (in parallel), then nvcc links
the shared library.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtslb.so")
LIB_CHECKED = os.path.join(HERE, "libtslb_checked.so")
LIB_HOSTSAN = os.path.join(HERE, "libtslb_hostsan.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJDIR = os.path.join(HERE, "_build")

SOURCES = [
    "tslb_api.cu",
    "tslb_aux.cu",
    "tslb_step_direct.cu",
    "tslb_step_factored.cu",
    "tslb_step_factored_f32.cu",
    "tslb_step_factored_bf16.cu",
    "tslb_step_factored_bf16sr.cu",
    "tslb_step_factored_f16.cu",
    "tslb_step_factored_f16sr.cu",
    "tslb_adjoint.cu",
    "tslb_noalloc.cu",
    "tslb_step2d.cu",
]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-Xptxas", "-v",
]

VARIANTS = {LIB: [], LIB_CHECKED: ["-DTSLB_CHECKED"]}
# Host code under AddressSanitizer / UndefinedBehaviorSanitizer (device code
# unchanged); built on demand by the CPU test of the ABI's host paths and
# selected with TSLB_HOSTSAN=1 (the process must preload the ASan runtime).
HOSTSAN_FLAGS = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined",
                 "-Xcompiler", "-fno-omit-frame-pointer"]  # one flag each: nvcc splits -Xcompiler at commas


def _stale(lib):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tslb.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(nvcc, src, obj, defs):
    cmd = [nvcc] + NVCC_FLAGS + defs + ["-I", INCLUDE, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.returncode, src, r.stdout + r.stderr


def build(force=False, verbose=False, variants=None):
    """Compile csrc/*.cu into libtslb.so and libtslb_checked.so next to this
    file (each only when out of date unless force).  Returns the product path.
    variants: a {library path: extra nvcc flags} map to build instead."""
    variants = VARIANTS if variants is None else variants
    todo = [lib for lib in variants if force or _stale(lib)]
    if not todo:
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJDIR, exist_ok=True)
    jobs = []
    for lib in todo:
        tag = os.path.splitext(os.path.basename(lib))[0]
        for s in SOURCES:
            obj = os.path.join(OBJDIR, "%s.%s.o" % (tag, os.path.splitext(s)[0]))
            jobs.append((lib, os.path.join(CSRC, s), obj))
    workers = max(1, min(len(jobs), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(lambda j: _compile(nvcc, j[1], j[2], variants[j[0]]), jobs))
    for rc, src, log in results:
        if rc != 0:
            sys.stderr.write(log)
            raise RuntimeError("nvcc failed compiling %s" % os.path.basename(src))
        if verbose:
            sys.stderr.write(log)
    for lib in todo:
        objs = [j[2] for j in jobs if j[0] == lib]
        link_extra = HOSTSAN_FLAGS if variants[lib] == HOSTSAN_FLAGS else []
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC"] + link_extra + ["-o", lib + ".tmp"]
                           + objs, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed linking %s" % os.path.basename(lib))
        os.replace(lib + ".tmp", lib)
    return LIB


def build_hostsan():
    """libtslb_hostsan.so: the library with its host code sanitized."""
    build(variants={LIB_HOSTSAN: HOSTSAN_FLAGS})
    return LIB_HOSTSAN


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
