"""Input generators: the rigid transform of a map and the two-agent
alignment workload (checked against scipy's rotation algebra)."""
import numpy as np

from paper_2412_09723_gb300 import scenes


def test_transform_scene_matches_scipy_rotation():
    from scipy.spatial.transform import Rotation

    sc = scenes.scene_uniform(300, 5).astype(np.float64)
    T = scenes.perturbed_w2c(12, 0.4, 70.0).astype(np.float64)
    out = scenes.transform_scene(sc, T)
    np.testing.assert_allclose(out.mean, sc.mean @ T[:3, :3].T + T[:3, 3], atol=2e-6)
    want = Rotation.from_matrix(T[:3, :3]) * Rotation.from_quat(sc.quat[:, [1, 2, 3, 0]])
    got = Rotation.from_quat(out.quat[:, [1, 2, 3, 0]].astype(np.float64))
    assert np.max((want.inv() * got).magnitude()) < 1e-5
    # rotation by R of a unit quaternion keeps its norm
    np.testing.assert_allclose(np.linalg.norm(out.quat, axis=1), np.linalg.norm(sc.quat, axis=1), rtol=1e-5)


def test_quaternion_of_rotation_all_branches():
    from scipy.spatial.transform import Rotation

    for ang, axis in [(10.0, (0, 0, 1)), (179.0, (1, 0, 0)), (179.0, (0, 1, 0)), (179.0, (0, 0, 1)),
                      (120.0, (1, 1, 1))]:
        R = Rotation.from_rotvec(np.radians(ang) * np.asarray(axis, float) / np.linalg.norm(axis)).as_matrix()
        q = scenes._quat_of_rotation(R)
        np.testing.assert_allclose(Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix(), R, atol=1e-12)


def test_alignment_workload_relation():
    a, b, perm, T_true, kfs, T0, cam = scenes.workload_alignment(n=5000, n_views=8)
    assert a.n == b.n == 5000 and len(kfs) == 8
    back = scenes.transform_scene(b, T_true.astype(np.float64))
    d = np.linalg.norm(back.mean - a.mean[perm], axis=1)
    assert np.sqrt(np.mean(d ** 2)) < 0.005 and np.max(d) < 0.03  # 2 mm jitter per axis
    assert np.max(np.abs(back.rgb - a.rgb[perm])) <= 0.1
    # the start is 1 cm / 0.5 degrees off T_true
    E = T0.astype(np.float64) @ np.linalg.inv(T_true.astype(np.float64))
    assert abs(np.linalg.norm(E[:3, 3]) - 0.01) < 1e-3
    ang = np.degrees(np.arccos(np.clip((np.trace(E[:3, :3]) - 1) / 2, -1, 1)))
    assert abs(ang - 0.5) < 0.02
