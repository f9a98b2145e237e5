"""The oracle's pins are sharp: each plausible slip, planted in a temporary
copy of the oracle source (CPU only), makes at least one pin fail."""
import ctypes
import importlib.util
import os
import subprocess

import pytest

import tests.test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name -> (exact text in the oracle, planted replacement)
MUTATIONS = {
    "background term dropped from dalpha": (
        "da += b.T * S * (gA - bgdot);", "da += b.T * S * (gA);"),
    "camera rotation transposed in J W": (
        "p.J[3 * i + 0] * k.R[0 + j] + p.J[3 * i + 1] * k.R[3 + j] + p.J[3 * i + 2] * k.R[6 + j]",
        "p.J[3 * i + 0] * k.R[3 * j] + p.J[3 * i + 1] * k.R[3 * j + 1] + p.J[3 * i + 2] * k.R[3 * j + 2]"),
    "clamped x' treated as constant in z": (
        "else dmc[2] += p.clx * p.limx * dxcl;", "else dmc[2] += 0;"),
    "conic off-diagonal sign": (
        "p.conic[1] = -p.cov[1] / det;", "p.conic[1] = p.cov[1] / det;"),
    "one quaternion partial sign": (
        "{2 * qy, 2 * qz, 2 * w, 2 * qx},     // 2(xz + wy)",
        "{2 * qy, 2 * qz, 2 * w, -2 * qx},     // 2(xz + wy)"),
    "pose rotation term sign": (
        "pose[3] += Wc[1] * dWc[2] - Wc[2] * dWc[1];", "pose[3] -= Wc[1] * dWc[2] - Wc[2] * dWc[1];"),
    "tile rectangle end": (
        "p.rect[2] = (int)i1 / kTile + 1;", "p.rect[2] = (int)(i1 + 1) / kTile + 1;"),
    "suffix sum without (1 - alpha)": (
        "Bd = b.alpha * depth[g] + (1 - b.alpha) * Bd;", "Bd = b.alpha * depth[g] + Bd;"),
    "stop test after blending": (
        "if (Tn < kTStop) break;\n    out.push_back({g, alpha, G, clamped, T, dx, dy});",
        "out.push_back({g, alpha, G, clamped, T, dx, dy});\n    if (Tn < kTStop) break;"),
    "depth order reversed": (
        "std::sort(items.begin(), items.end());",
        "std::sort(items.begin(), items.end(), [](const auto& a, const auto& b) {"
        " return std::make_tuple(std::get<0>(a), -std::get<1>(a), std::get<2>(a)) <"
        " std::make_tuple(std::get<0>(b), -std::get<1>(b), std::get<2>(b)); });"),
    "low-pass filter dropped": (
        "p.cov[0] = c2[0] + kLowPass;", "p.cov[0] = c2[0];"),
    "visibility from T behind instead of in front": (
        "for (const Blend& b : bl) mine[b.g] = std::max(mine[b.g], b.T);",
        "for (const Blend& b : bl) mine[b.g] = std::max(mine[b.g], b.T * (1 - b.alpha));"),
}


def _load_mutant(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "gsff_oracle.cpp")).read()
    assert src.count(old) == 1, name
    cpp = tmp_path / "mut.cpp"
    so = tmp_path / "mut.so"
    cpp.write_text(src.replace(old, new))
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", str(cpp), "-o",
                    str(so)], check=True, capture_output=True)
    spec = importlib.util.spec_from_file_location("oracle_mutant", os.path.join(ROOT, "oracle", "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    lib = ctypes.CDLL(str(so))
    lib.ora_bin.restype = ctypes.c_int64
    lib.ora_num_threads.restype = ctypes.c_int
    mod._lib = lib
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, sg, name):
    old, new = MUTATIONS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    failed = []
    for tname in sorted(n for n in dir(pins) if n.startswith("test_")):
        try:
            getattr(pins, tname)(mut, sg)
        except AssertionError:
            failed.append(tname)
    assert failed, f"no pin caught: {name}"


# planted slips in the tracking pieces, caught by tests/test_oracle_tracking.py
TRACKING_MUTATIONS = {
    "pose update applied on the right": (
        "for (int k = 0; k < 3; ++k) sum += Rd[3 * i + k] * R[3 * k + j];",
        "for (int k = 0; k < 3; ++k) sum += R[3 * i + k] * Rd[3 * k + j];"),
    "V matrix dropped from the translation": (
        "for (int i = 0; i < 3; ++i) td[i] = V[3 * i] * dl[0] + V[3 * i + 1] * dl[1] + V[3 * i + 2] * dl[2];",
        "for (int i = 0; i < 3; ++i) td[i] = dl[i];"),
    "Sobel without the 1/8 normalisation": (
        "const float gx = (a - b) * 0.125f, gy = (c - d) * 0.125f;",
        "const float gx = (a - b), gy = (c - d);"),
    "Adam step sign": (
        "dl[i] = -(i < 3 ? lr_t : lr_r) * mh / (std::sqrt(vh) + eps);",
        "dl[i] = (i < 3 ? lr_t : lr_r) * mh / (std::sqrt(vh) + eps);"),
}


@pytest.mark.parametrize("name", sorted(TRACKING_MUTATIONS))
def test_tracking_pins_catch_planted_mistake(tmp_path, name):
    import inspect

    import tests.test_oracle_tracking as tpins
    old, new = TRACKING_MUTATIONS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    failed = []
    for tname in sorted(n for n in dir(tpins) if n.startswith("test_")):
        fn = getattr(tpins, tname)
        kw = {"scale": 1.0} if "scale" in inspect.signature(fn).parameters else {}
        try:
            fn(mut, **kw)
        except AssertionError:
            failed.append(tname)
    assert failed, f"no pin caught: {name}"


# planted slips in the semantic pieces, caught by tests/test_oracle_semantic.py
SEMANTIC_MUTATIONS = {
    "cross-entropy gradient without 1/HW": (
        "grad[at(p, c)] = (std::exp(F[at(p, c)] - mx) / sum - (c == lab ? 1.0 : 0.0)) / (double)HW;",
        "grad[at(p, c)] = (std::exp(F[at(p, c)] - mx) / sum - (c == lab ? 1.0 : 0.0));"),
    "cross-entropy sign": (
        "loss += (mx + std::log(sum) - F[at(p, lab)]) / (double)HW;",
        "loss += (F[at(p, lab)] - mx - std::log(sum)) / (double)HW;"),
    "logits with a separate multiply and add": (
        "for (int c = 0; c < M; ++c) acc = std::fmaf(f[p * M + c], q[(size_t)l * M + c], acc);",
        "for (int c = 0; c < M; ++c) { const float pr = f[p * M + c] * q[(size_t)l * M + c]; acc = acc + pr; }"),
    "label probabilities not normalised": (
        "for (int l = 0; l < L; ++l) probs[p * L + l] = std::exp(z[l] - mx) / sum;",
        "for (int l = 0; l < L; ++l) probs[p * L + l] = std::exp(z[l] - mx);"),
}


@pytest.mark.parametrize("name", sorted(SEMANTIC_MUTATIONS))
def test_semantic_pins_catch_planted_mistake(tmp_path, name):
    import tests.test_oracle_semantic as spins
    old, new = SEMANTIC_MUTATIONS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    failed = []
    for tname in sorted(n for n in dir(spins) if n.startswith("test_")):
        try:
            getattr(spins, tname)(mut)
        except AssertionError:
            failed.append(tname)
    assert failed, f"no pin caught: {name}"


# planted slips in the spherical-harmonic colour, caught by tests/test_oracle_sh.py
SH_MUTATIONS = {
    "camera centre sign": (
        "for (int i = 0; i < 3; ++i) C[i] = -(R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]);",
        "for (int i = 0; i < 3; ++i) C[i] = (R[i] * t[0] + R[3 + i] * t[1] + R[6 + i] * t[2]);"),
    "sqrt2 dropped for m != 0": (
        "Y[l * l + l + m] = (std::sqrt(2.0) * N) * (P[l] * re[m]);",
        "Y[l * l + l + m] = N * (P[l] * re[m]);"),
    "Legendre recurrence coefficient": (
        "P[l] = (1.0 / (l - m)) * ((double)(2 * l - 1) * (z * P[l - 1]) - (double)(l + m - 1) * P[l - 2]);",
        "P[l] = (1.0 / (l - m)) * ((double)(2 * l - 1) * (z * P[l - 1]) - (double)(l + m) * P[l - 2]);"),
    "pose gradient without R": (
        "for (int i = 0; i < 3; ++i) d_pose[i] += R[3 * i] * sum_dmu[0] + R[3 * i + 1] * sum_dmu[1] + R[3 * i + 2] * sum_dmu[2];",
        "for (int i = 0; i < 3; ++i) d_pose[i] += sum_dmu[i];"),
}


@pytest.mark.parametrize("name", sorted(SH_MUTATIONS))
def test_sh_pins_catch_planted_mistake(tmp_path, sg, name):
    import inspect

    import tests.test_oracle_sh as shpins
    old, new = SH_MUTATIONS[name]
    mut = _load_mutant(tmp_path, name, old, new)
    failed = []
    for tname in sorted(n for n in dir(shpins) if n.startswith("test_")):
        fn = getattr(shpins, tname)
        kw = {"sg": sg} if "sg" in inspect.signature(fn).parameters else {}
        try:
            fn(mut, **kw)
        except AssertionError:
            failed.append(tname)
    assert failed, f"no pin caught: {name}"
