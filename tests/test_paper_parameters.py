"""The workloads use the transport parameters and timing-case geometry that
GPUMCD states for its runs (Sec. III; tests/golden/paper_parameters.json)."""
import json
import os

import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_parameters.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as f:
        return {k: v["value"] for k, v in json.load(f).items() if not k.startswith("_")}


def test_cutoffs_and_step_parameter(paper):
    ph = W.DEFAULT_PHYSICS
    assert ph.p_cut == paper["photon_cutoff_mev"]
    assert ph.estepe == paper["estepe"]
    # E_cut is a total energy; the electron cut-off here is kinetic and rounds
    # 0.7 - m_e c^2 = 0.189 MeV to 0.2 MeV
    kinetic = paper["electron_cutoff_total_mev"] - paper["electron_rest_energy_mev"]
    assert ph.e_abs == pytest.approx(kinetic, abs=0.015)


def test_timing_case_beams(paper):
    for particle, key in ((W.ELECTRON, "electron_histories"), (W.PHOTON, "photon_histories")):
        plan = W.config2(particle)
        assert plan.n_histories == paper[key]
        assert plan.source.energy == paper["beam_energy_mev"]
        assert plan.source.spectrum_edges is None and plan.source.beam == W.BEAM_SQUARE


def test_timing_case_phantom_extent(paper):
    # 128^3 voxels of 0.25 cm cover the paper's 64^3 grid of 0.5 cm voxels
    ph = W.config2(W.ELECTRON).phantom
    extent = paper["phantom_voxels_per_axis"] * paper["voxel_cm"]
    assert all(e == pytest.approx(extent) for e in ph.extent_cm)
    assert W.config2(W.ELECTRON, n=64, voxel_cm=0.5).phantom.dims == (64, 64, 64)
