"""The serving loop's submission lock (host logic, no GPU): batch submissions
hold it together, a slice update alone; an update waits for the submissions in
progress, and a waiting update lets no new submission in before it."""
import threading
import time

from paper_2409_07759_b300.serving import _SharedLock


def test_shared_holders_run_together():
    lk = _SharedLock()
    inside = []
    both = threading.Barrier(2, timeout=5)

    def sub():
        lk.acquire_shared()
        try:
            inside.append(1)
            both.wait()  # both holders inside at once, or this times out
        finally:
            lk.release_shared()

    th = [threading.Thread(target=sub) for _ in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(5)
    assert len(inside) == 2


def test_update_waits_for_submissions_and_blocks_new_ones():
    lk = _SharedLock()
    log = []
    lk.acquire_shared()  # a submission in progress

    def update():
        lk.acquire_exclusive()
        log.append("update")
        lk.release_exclusive()

    def late_submission():
        lk.acquire_shared()
        log.append("late")
        lk.release_shared()

    up = threading.Thread(target=update)
    up.start()
    time.sleep(0.1)
    assert log == []  # the update waits for the submission in progress
    late = threading.Thread(target=late_submission)
    late.start()
    time.sleep(0.1)
    assert log == []  # the late submission waits behind the waiting update
    lk.release_shared()
    up.join(5)
    late.join(5)
    assert log == ["update", "late"]
